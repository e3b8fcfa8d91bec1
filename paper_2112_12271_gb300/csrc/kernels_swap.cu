// kernels_swap.cu -- SWAP Monte Carlo diameter exchanges (Sec. II.D).
//
// The paper draws pN candidate pairs, builds full neighbour lists for the
// chosen atoms in parallel ("buildNLs"), then runs the exchanges serially on
// one thread.  Here the exchanges run in parallel and give the serial
// answer: pair k may run once no earlier pending pair writes an atom that k
// reads (its two atoms and their neighbours) -- the same relation in the
// other direction because neighbour sets are symmetric.  Each round every
// pending pair claims its two atoms with an atomicMin of (round tag, k);
// a pair whose read set holds no claim from an earlier pair of this round
// executes.  The lowest pending pair always runs, so the rounds end.
//
// Energies (Eqs. (10)-(11)): E_b sums U(sigma_i, sigma_b, r_ib) over the
// neighbours b of i except j, plus the same for j; E_a exchanges sigma_i
// and sigma_j.  The neighbour lists hold every atom closer than the largest
// diameter (no pair can interact beyond it, whatever the exchange), found
// over the 3^d linked subcells of the last build.  Metropolis acceptance
// u < exp(-(E_a - E_b)/T) in FP64; an accepted exchange swaps sigma and
// mass and rescales both velocities by sqrt(m_old/m_new).
#include "launch.h"

namespace hdmd {
namespace {

constexpr int NT = 256;

// Philox4x32-10 (Salmon et al., SC'11): two multiply-xor lanes per round,
// key advanced by the Weyl constants between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

__global__ void k_swap_draw(SwapDev sw, uint64_t seed, int sweep, int N) {
    const int p = blockIdx.x * NT + threadIdx.x;
    if (p >= sw.npairs) return;
    uint32_t c[4] = {(uint32_t)p, (uint32_t)sweep, 0x53574150u, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    int i = (int)(((uint64_t)c[0] * (uint64_t)N) >> 32);
    int j = (int)(((uint64_t)c[1] * (uint64_t)(N - 1)) >> 32);
    if (j >= i) ++j;
    const uint64_t bits = ((uint64_t)c[3] << 32) | c[2];
    sw.ids[2 * p] = i;
    sw.ids[2 * p + 1] = j;
    sw.u[p] = (double)(bits >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void k_slot_of(Dev dv, SwapDev sw) {
    const int s = blockIdx.x * NT + threadIdx.x;
    if (s < dv.N) sw.slot_of[dv.id[s]] = s;
}

__global__ void k_pairs(SwapDev sw) {
    const int p = blockIdx.x * NT + threadIdx.x;
    if (p >= sw.npairs) return;
    sw.pairs[2 * p] = sw.slot_of[sw.ids[2 * p]];
    sw.pairs[2 * p + 1] = sw.slot_of[sw.ids[2 * p + 1]];
    sw.state[p] = 0;
}

// swap lists: warp per candidate atom, over the linked subcells of its
// build-time subcell, FP32 cell-relative rows of buffer buf (current x)
template <int D, bool WRAP>
__global__ void k_swap_lists(Dev dv, SwapDev sw, int buf) {
    constexpr int RF = Rows<D>::RF;
    const int w = (blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= 2 * sw.npairs) return;
    const int a = sw.pairs[w];
    const float *ra = dv.gs[buf] + (size_t)a * RF;
    float xa[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xa[k] = ra[k];
    const int n = dv.n;
    int C[D];
    {
        int t = dv.cellid[a];
        for (int k = D - 1; k >= 0; --k) { C[k] = t % n; t /= n; }
    }
    const float Lsc = dv.Lsc_f, hL = dv.halfL_f;
    const float R = (float)sw.rcut * (1.0f + 1e-5f) + 1e-5f;
    const float R2 = R * R;
    const int base = WRAP ? 3 : (n == 1 ? 1 : 2);
    const int S = pow_int(base, D);
    int cnt = 0;
    int32_t *out = sw.slist + (size_t)w * sw.scap;
    for (int s = 0; s < S; ++s) {
        int rem = s, J = 0;
        int off[D];
        for (int k = D - 1; k >= 0; --k) { off[k] = rem % base - (WRAP ? 1 : 0); rem /= base; }
        for (int k = 0; k < D; ++k) {
            int cj = C[k] + off[k];
            cj = cj < 0 ? cj + n : (cj >= n ? cj - n : cj);
            J = J * n + cj;
        }
        const int b0 = dv.cell_start[J], b1 = dv.cell_start[J + 1];
        for (int bb = b0; bb < b1; bb += 32) {
            const int b = bb + lane;
            bool hit = false;
            if (b < b1 && b != a) {
                const float *rb = dv.gs[buf] + (size_t)b * RF;
                float r2 = 0.f;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    float dx;
                    if (WRAP) {
                        dx = fmaf((float)off[k], Lsc, rb[k]) - xa[k];
                    } else {
                        dx = rb[k] - xa[k];
                        if (off[k]) {
                            const float dp = (rb[k] + Lsc) - xa[k];
                            dx = dp > hL ? (rb[k] - Lsc) - xa[k] : dp;
                        } else if (n == 1) {
                            if (dx > hL) dx = (rb[k] - Lsc) - xa[k];
                            else if (dx < -hL) dx = (rb[k] + Lsc) - xa[k];
                        }
                    }
                    r2 = fmaf(dx, dx, r2);
                }
                hit = r2 < R2;
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int idx = cnt + __popc(m & ((1u << lane) - 1u));
                if (idx < sw.scap) out[idx] = b;
            }
            cnt += __popc(m);
        }
    }
    if (lane == 0) {
        sw.scount[w] = min(cnt, sw.scap);
        if (cnt > sw.scap) atomicMax(sw.overflow, cnt);
    }
}

__device__ __forceinline__ unsigned long long round_tag(unsigned round) {
    return (unsigned long long)(0xFFFFFFFEu - round) << 32;
}

__global__ void k_swap_claim(SwapDev sw, unsigned round) {
    const int p = blockIdx.x * NT + threadIdx.x;
    if (p >= sw.npairs || sw.state[p] != 0) return;
    const unsigned long long v = round_tag(round) | (unsigned)p;
    atomicMin(&sw.owner[sw.pairs[2 * p]], v);
    atomicMin(&sw.owner[sw.pairs[2 * p + 1]], v);
}

// pair energy of diameters si, sj at distance r under the system's law
// (harmonic or the Morse law of Eq. (1); prefactor eps or, volume-scaled,
// eps (si sj)^(D/2))
template <int D>
__device__ __forceinline__ double pair_u(const Dev &dv, double r, double si, double sj) {
    const double s = 0.5 * (si + sj);
    if (r >= s) return 0.0;
    double e = dv.eps;
    if (dv.eps_scale) {
        const double p = si * sj;
        double q = 1.0;
#pragma unroll
        for (int k = 0; k < D / 2; ++k) q *= p;
        if (D & 1) q *= sqrt(p);
        e *= q;
    }
    if (dv.law == 1) {
        const double m = expm1(-dv.morse_a * (r - s));
        return e * m * m;
    }
    if (dv.law == 2) {
        double q = 1.0, b = s / r;
        for (int n = dv.mie_n; n; n >>= 1, b *= b)
            if (n & 1) q *= b;
        return e * (q - 1.0) * (q - 1.0);
    }
    const double g = 1.0 - r / s;
    return 0.5 * e * g * g;
}

// FP64 distance of atoms a and b at the current positions x0 + dlt
template <int D>
__device__ __forceinline__ double dist64(const Dev &dv, int a, int b) {
    double r2 = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const size_t oa = (size_t)k * dv.Npad + a, ob = (size_t)k * dv.Npad + b;
        double dx = (dv.x0[ob] + dv.dlt[ob]) - (dv.x0[oa] + dv.dlt[oa]);
        dx -= dv.L * rint(dx * dv.invL);
        r2 += dx * dx;
    }
    return sqrt(r2);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int D>
__global__ void k_swap_exec(Dev dv, SwapDev sw, unsigned round) {
    const int p = (blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= sw.npairs) return;
    if (sw.state[p] != 0) return;            // warp-uniform
    const int i = sw.pairs[2 * p], j = sw.pairs[2 * p + 1];
    const unsigned long long tag = round_tag(round);
    const int ni = sw.scount[2 * p], nj = sw.scount[2 * p + 1];
    const int32_t *Si = sw.slist + (size_t)(2 * p) * sw.scap;
    const int32_t *Sj = sw.slist + (size_t)(2 * p + 1) * sw.scap;
    // read set: i, j, S(i), S(j); blocked by a claim of an earlier pair
    bool ok = true;
    for (int t = lane; t < ni + nj + 2; t += 32) {
        const int a = t == 0 ? i : (t == 1 ? j : (t - 2 < ni ? Si[t - 2] : Sj[t - 2 - ni]));
        const unsigned long long o = sw.owner[a];
        if ((o & 0xFFFFFFFF00000000ull) == tag && (unsigned)(o & 0xFFFFFFFFu) < (unsigned)p) ok = false;
    }
    if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicAdd(sw.npend, 1);
        return;
    }
    const double si = dv.sigma[i], sj = dv.sigma[j];
    double eb = 0.0, ea = 0.0;
    for (int t = lane; t < ni; t += 32) {
        const int b = Si[t];
        if (b == j) continue;
        const double r = dist64<D>(dv, i, b), sb = dv.sigma[b];
        eb += pair_u<D>(dv, r, si, sb);
        ea += pair_u<D>(dv, r, sj, sb);
    }
    for (int t = lane; t < nj; t += 32) {
        const int b = Sj[t];
        if (b == i) continue;
        const double r = dist64<D>(dv, j, b), sb = dv.sigma[b];
        eb += pair_u<D>(dv, r, sj, sb);
        ea += pair_u<D>(dv, r, si, sb);
    }
    eb = warp_sum(eb);
    ea = warp_sum(ea);
    const bool acc = sw.u[p] < exp(-(ea - eb) / sw.T);
    if (acc) {
        // each lane may touch one coordinate of the two velocities
        if (dv.inv_mass) {
            const double imi = dv.inv_mass[i], imj = dv.inv_mass[j];
            const double fi = sqrt(imj / imi), fj = sqrt(imi / imj);   // sqrt(m_i / m_j), sqrt(m_j / m_i)
            for (int k = lane; k < D; k += 32) {
                dv.v[(size_t)k * dv.Npad + i] *= fi;
                dv.v[(size_t)k * dv.Npad + j] *= fj;
            }
            __syncwarp();
            if (lane == 0) { dv.inv_mass[i] = imj; dv.inv_mass[j] = imi; }
        }
        if (lane == 0) { dv.sigma[i] = sj; dv.sigma[j] = si; }
    }
    if (lane == 0) {
        sw.state[p] = acc ? 2 : 1;
        if (acc) atomicAdd(sw.nacc, 1ull);
    }
}

template <int D>
void prepare_impl(const Dev &dv, const SwapDev &sw, int buf, cudaStream_t s) {
    k_slot_of<<<(dv.N + NT - 1) / NT, NT, 0, s>>>(dv, sw);
    k_pairs<<<(sw.npairs + NT - 1) / NT, NT, 0, s>>>(sw);
    const int warps = 2 * sw.npairs;
    const int blocks = (warps * 32 + NT - 1) / NT;
    if (dv.n >= 3) k_swap_lists<D, true><<<blocks, NT, 0, s>>>(dv, sw, buf);
    else k_swap_lists<D, false><<<blocks, NT, 0, s>>>(dv, sw, buf);
}

template <int D>
void round_impl(const Dev &dv, const SwapDev &sw, unsigned round, cudaStream_t s) {
    k_swap_claim<<<(sw.npairs + NT - 1) / NT, NT, 0, s>>>(sw, round);
    k_swap_exec<D><<<(sw.npairs * 32 + NT - 1) / NT, NT, 0, s>>>(dv, sw, round);
}

}  // namespace

void launch_swap_draw(const SwapDev &sw, uint64_t seed, int sweep, int N, cudaStream_t s) {
    k_swap_draw<<<(sw.npairs + NT - 1) / NT, NT, 0, s>>>(sw, seed, sweep, N);
}

void launch_swap_prepare(const Dev &dv, const SwapDev &sw, int buf, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, prepare_impl, dv, sw, buf, s);
}

void launch_swap_round(const Dev &dv, const SwapDev &sw, unsigned round, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, round_impl, dv, sw, round, s);
}

}  // namespace hdmd
