// kernels_nbr.cu -- full Verlet lists over the 3^d linked subcells
// (Sec. II.C, Fig. 1).
//
// As in the paper the work is organised by home subcell, the linked subcells
// are enumerated on the fly from a base-3 counter (never stored), and the
// atom double loop is innermost.  On the GPU:
//   - one warp owns a batch of up to H atoms of one home subcell (their
//     coordinates and radii live in registers of every lane), so a subcell
//     holding many atoms is split over several warps;
//   - the stencil is walked as 3^(d-1) "rows": the three subcells that differ
//     only along the last axis are adjacent in the linear index of Eq. (9),
//     so after the counting sort their atoms form one contiguous range (two
//     when the row wraps around the box), read with coalesced row loads, one
//     candidate per lane;
//   - before a row is read each home atom tests the distance from itself to
//     the row's box; only home atoms that can reach it test its candidates;
//   - each home atom's hits are compacted with __ballot_sync/__popc, so the
//     lists come out in the same order on every run;
//   - a pair is kept iff r^2 < (sigma_ij + s)^2.  The FP32 distance
//     (cell-relative coordinates, error ~1e-7) decides unless r^2 lies in a
//     guard band around the cutoff, where the FP64 distance decides, so the
//     lists equal those of an all-FP64 search.
// With n_cell = 2 the offsets -1 and +1 name the same subcell, so each
// subcell is visited once (offsets {0, +1}) and every pair takes the minimum
// image along the axes where the two subcells differ; the paper switches to
// an all-pairs search there, which this amounts to.
#include "launch.h"

namespace hdmd {
namespace {

constexpr int NT = 128;   // threads per block: 4 warps, one home batch each

template <int D, bool WRAP>
__global__ void __launch_bounds__(NT, 4) k_nbr_build(Dev dv, bool guarded) {
    if (guarded && *((volatile int *)&dv.flags->rebuild) == 0) return;
    constexpr int RF = Rows<D>::RF;
    constexpr int H = home_batch(D);
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * NT + threadIdx.x) >> 5;
    const int nbatch = dv.batch_start[dv.ncells];
    if (w >= nbatch) return;   // warp-uniform
    // home subcell: largest c with batch_start[c] <= w
    int lo = 0, hi = dv.ncells - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (dv.batch_start[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const int c = lo;
    const int cs = dv.cell_start[c], ce = dv.cell_start[c + 1];
    const int h0 = cs + (w - dv.batch_start[c]) * H;
    const int nh = min(H, ce - h0);
    const int n = dv.n;
    int C[D];
    {
        int t = c;
#pragma unroll
        for (int k = D - 1; k >= 0; --k) { C[k] = t % n; t /= n; }
    }
    const float Lsc = dv.Lsc_f, hLsc = 0.5f * dv.Lsc_f, hL = dv.halfL_f;
    const float skin = (float)dv.skin;
    const float band_abs = 1e-5f * Lsc * Lsc;

    // home atoms in registers (identical in every lane)
    float xh[H][D], rh[H];
    int cnt[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int i = h < nh ? h0 + h : h0;
        const float *ri = dv.gs0 + (size_t)i * RF;
#pragma unroll
        for (int k = 0; k < D; ++k) xh[h][k] = ri[k];
        rh[h] = ri[D] + skin;
        cnt[h] = 0;
    }
    const float reach_pad = dv.hmax_f;   // largest candidate radius
    // lane h (< nh) keeps its own home atom for the row-reach test
    float xmine[D];
    float reach2_mine = -1.f;
    {
        const int i = lane < nh ? h0 + lane : h0;
        const float *ri = dv.gs0 + (size_t)i * RF;
#pragma unroll
        for (int k = 0; k < D; ++k) xmine[k] = ri[k];
        const float reach = (ri[D] + skin + reach_pad) * (1.0f + 1e-5f) + 1e-5f;
        if (lane < nh) reach2_mine = reach * reach;
    }

    const int base = WRAP ? 3 : 2;
    const int Srow = pow_int(base, D - 1);
    int Jstride = 1;   // n^(D-1) is not needed: rows differ in axes 0..D-2
    (void)Jstride;
    const int cl = C[D - 1];
    for (int sr = 0; sr < Srow; ++sr) {
        // offsets of axes 0..D-2 from the base-3 (or base-2) digits of sr
        int off[D];
        {
            int rem = sr;
#pragma unroll
            for (int k = D - 2; k >= 0; --k) { off[k] = rem % base - (WRAP ? 1 : 0); rem /= base; }
        }
        int Jrow = 0;   // linear index of the row's subcell with last coordinate 0
#pragma unroll
        for (int k = 0; k < D - 1; ++k) {
            int cj = C[k] + off[k];
            cj = cj < 0 ? cj + n : (cj >= n ? cj - n : cj);
            Jrow = Jrow * n + cj;
        }
        Jrow *= n;
        // which home atoms can reach this row
        unsigned active;
        if (WRAP) {
            float b2 = 0.f;
#pragma unroll
            for (int k = 0; k < D - 1; ++k) {
                float dk = off[k] > 0 ? hLsc - xmine[k] : (off[k] < 0 ? xmine[k] + hLsc : 0.f);
                dk = fmaxf(dk, 0.f);
                b2 = fmaf(dk, dk, b2);
            }
            active = __ballot_sync(0xffffffffu, b2 < reach2_mine) & ((1u << H) - 1u);
        } else {
            active = (1u << nh) - 1u;
        }
        if (!active) continue;
        uint32_t rowcode = 0;
#pragma unroll
        for (int k = 0; k < D - 1; ++k) rowcode |= (uint32_t)(off[k] + 1) << (2 * k);
        // candidate ranges of the row: up to two contiguous pieces
        int ra0, ra1, rb0 = 0, rb1 = 0;
        if (WRAP) {
            const int cm = cl - 1, cp = cl + 1;
            if (cm >= 0 && cp < n) {
                ra0 = dv.cell_start[Jrow + cm];
                ra1 = dv.cell_start[Jrow + cp + 1];
            } else if (cm < 0) {   // cells 0, 1 then n-1
                ra0 = dv.cell_start[Jrow];
                ra1 = dv.cell_start[Jrow + min(cp, n - 1) + 1];
                rb0 = dv.cell_start[Jrow + n - 1];
                rb1 = dv.cell_start[Jrow + n];
                if (n - 1 <= cp) rb0 = rb1;   // n == 2 cannot occur here (n >= 3)
            } else {               // cells n-2, n-1 then 0
                ra0 = dv.cell_start[Jrow + cm];
                ra1 = dv.cell_start[Jrow + n];
                rb0 = dv.cell_start[Jrow];
                rb1 = dv.cell_start[Jrow + 1];
            }
        } else {
            ra0 = dv.cell_start[Jrow];
            ra1 = dv.cell_start[Jrow + 2];
        }
        for (int piece = 0; piece < 2; ++piece) {
            const int p0 = piece ? rb0 : ra0, p1 = piece ? rb1 : ra1;
            for (int b0 = p0; b0 < p1; b0 += 32) {
                const int j = b0 + lane;
                const bool okj = j < p1;
                const int jj = okj ? j : p0;
                // last-axis subcell of the candidate -> its offset
                int olast;
                {
                    const int cjl = dv.cellid[jj] - Jrow;   // 0..n-1
                    int o = cjl - cl;
                    if (WRAP) o = o > 1 ? o - n : (o < -1 ? o + n : o);
                    else o = o != 0 ? 1 : 0;
                    olast = o;
                }
                float rj[RF];
                {
                    const float4 *rj4 = reinterpret_cast<const float4 *>(dv.gs0 + (size_t)jj * RF);
#pragma unroll
                    for (int q = 0; q < RF / 4; ++q) {
                        const float4 t = __ldg(rj4 + q);
                        rj[4 * q] = t.x; rj[4 * q + 1] = t.y; rj[4 * q + 2] = t.z; rj[4 * q + 3] = t.w;
                    }
                }
                if (WRAP) {
#pragma unroll
                    for (int k = 0; k < D - 1; ++k) rj[k] = fmaf((float)off[k], Lsc, rj[k]);
                    rj[D - 1] = fmaf((float)olast, Lsc, rj[D - 1]);
                }
                const uint32_t wcode = WRAP ? (rowcode | ((uint32_t)(olast + 1) << (2 * (D - 1)))) : 0u;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    if (!(active & (1u << h))) continue;   // warp-uniform
                    const int i = h0 + h;
                    bool hit = false;
                    uint32_t code = wcode;
                    if (okj && j != i) {
                        float r2 = 0.f;
                        if (WRAP) {
#pragma unroll
                            for (int k = 0; k < D; ++k) {
                                const float dx = rj[k] - xh[h][k];
                                r2 = fmaf(dx, dx, r2);
                            }
                        } else {
                            code = 0u;
#pragma unroll
                            for (int k = 0; k < D; ++k) {
                                const int ok = k < D - 1 ? off[k] : olast;   // 0 or +1
                                float dx = rj[k] - xh[h][k];
                                int o = ok;
                                if (ok) {
                                    const float dp = (rj[k] + Lsc) - xh[h][k];
                                    if (dp > hL) { dx = (rj[k] - Lsc) - xh[h][k]; o = -1; }
                                    else dx = dp;
                                }
                                code |= (uint32_t)(o + 1) << (2 * k);
                                r2 = fmaf(dx, dx, r2);
                            }
                        }
                        const float rc = rh[h] + rj[D];
                        const float rc2 = rc * rc;
                        const float diff = r2 - rc2;
                        const float band = band_abs + 1e-5f * rc2;
                        if (diff > band) {
                            hit = false;
                        } else if (fabsf(diff) <= band) {
                            // FP64 decision (positions are x0 at a build)
                            double s2 = 0.0;
                            for (int k = 0; k < D; ++k) {
                                double dx = dv.x0[(size_t)k * dv.Npad + j] - dv.x0[(size_t)k * dv.Npad + i];
                                dx -= dv.L * rint(dx * dv.invL);
                                s2 += dx * dx;
                            }
                            const double rcd = 0.5 * (dv.sigma[i] + dv.sigma[j]) + dv.skin;
                            hit = s2 < rcd * rcd;
                        } else {
                            hit = diff < 0.f;
                        }
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, hit);
                    if (!m) continue;
                    if (hit) {
                        const int idx = cnt[h] + __popc(m & ((1u << lane) - 1u));
                        if (idx < dv.cap) {
                            const int64_t pos = list_pos(idx, i, dv.Npad, dv.G);
                            dv.nbr[pos] = j;
                            dv.code[pos] = code;
                        }
                    }
                    cnt[h] += __popc(m);
                }
            }
        }
    }
    if (lane < nh) {
        int cnt_l = 0;
#pragma unroll
        for (int h = 0; h < H; ++h) if (h == lane) cnt_l = cnt[h];
        const int i = h0 + lane;
        dv.nnbr[i] = min(cnt_l, dv.cap);
        if (cnt_l > dv.cap) atomicOr(&dv.flags->error, (int)ERR_OVERFLOW);
        atomicMax(&dv.flags->max_count, cnt_l);
        atomicAdd((unsigned long long *)&dv.flags->total_entries, (unsigned long long)cnt_l);
    }
}

template <int D>
void nbr_impl(const Dev &dv, bool guarded, cudaStream_t s) {
    // upper bound on the number of home batches: N / H + n_cells
    const int64_t warps = (int64_t)dv.N / home_batch(D) + dv.ncells + 1;
    const int blocks = (int)((warps * 32 + NT - 1) / NT);
    if (dv.n >= 3)
        k_nbr_build<D, true><<<blocks, NT, 0, s>>>(dv, guarded);
    else
        k_nbr_build<D, false><<<blocks, NT, 0, s>>>(dv, guarded);
}

}  // namespace

void launch_nbr_build(const Dev &dv, bool guarded, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, nbr_impl, dv, guarded, s);
}

}  // namespace hdmd
