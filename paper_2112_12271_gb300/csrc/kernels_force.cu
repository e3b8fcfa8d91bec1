// kernels_force.cu -- the pair force / energy / virial loop over the full
// Verlet list (Sec. II.B getforce) fused with the velocity-Verlet half kicks
// and drift (Sec. II.B leapfrog, kick-drift-kick), the displacement trigger
// of the list (Sec. II.C) and the FP64 reductions of the thermodynamic and
// FIRE scalars (Sec. II.B FIRE, Sec. II.E getthermo).
//
// Pair law: harmonic soft spheres or the Morse law of Eq. (1), see
// dev_force.cuh.  NVT: the Berendsen factor scales the second kick (the
// paper fuses its thermostat into that kick, Sec. II.B).
//
// Thread mapping: G consecutive lanes share one atom (G in 1..32); lane g
// walks list entries g, g+G, ... (coalesced thanks to the list layout), the
// partial forces meet through xor shuffles and lane 0 of the group does the
// per-atom epilogue.  FP32 pair arithmetic reads cell-relative FP32 rows
// (x_i - x_j = gs_i - gs_j - o Lsc with o from the entry's code); FP64 pair
// arithmetic reads absolute FP64 rows with the minimum image.  Positions,
// velocities and every global sum stay FP64; sums are reduced per block and
// folded in block order, so results repeat bit for bit.
//
// One MD step of KDK is  kick(F_n) drift -> [rebuild?] -> F_{n+1} kick(F_{n+1}).
// A launch with kick2 + kick1_drift does "F_n; kick(F_n); kick(F_n); drift",
// i.e. the end of step n-1 and the start of step n, reading the gather rows
// of x_n and writing those of x_{n+1} into the other buffer.
#include <type_traits>

#include "dev_fire.cuh"
#include "dev_force.cuh"

#ifndef HDMD_STEP_MIN_BLOCKS
#define HDMD_STEP_MIN_BLOCKS 8
#endif
#include "launch.h"

namespace hdmd {
namespace {

constexpr int NT = kStepNT;   // one wave of blocks at the benchmark size

// Displacement trigger, shared by the MD and FIRE update kernels: every
// block stores its max |dlt|^2 (float bits: non-negative floats order as
// unsigned integers, NaN above all) in a word of its own; the last block
// (ticket, no waiting) takes the maximum over all blocks and turns it into
// the rebuild flag and, inside a CUDA graph, into the IF condition.
// With a thermostat (nvt != 0) the same ticket also folds sum m v^2 of the
// thermostatted velocities (per-block partials at partials[maxblocks + b],
// summed in a fixed order) into the Berendsen factor of the next step:
// lambda = sqrt(1 + rate (T_target/T - 1)), T = sum m v^2 / (d (N - 1)).
__device__ __forceinline__ double block_sum_fixed(double a, double *ws) {
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = a;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    return t;   // valid in thread 0
}

// With rule 1 (the paper's, Sec. II.C) the trigger is evaluated after every
// n_bet-th MD step only and fires when at least 0.1 % of the atoms have moved
// by s/2 (blk_half: this block's count) or any atom by s.
__device__ __forceinline__ void trigger_fold(const Dev &dv, float blk_max_d2, bool blk_bad,
                                             unsigned long long cond, int nvt = 0,
                                             double kin = 0.0, double rate = 0.0,
                                             double T_target = 0.0, int rule = 0,
                                             int n_bet = 1, int blk_half = 0) {
    __shared__ bool last;
    __shared__ unsigned wmax[32];
    __shared__ unsigned whalf[32];
    __shared__ double wsum[32];
    unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(blk_max_d2));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = bits;
    if (blk_bad) atomicOr(&dv.flags->error, (int)ERR_LOST);
    __syncthreads();
    const double kblk = nvt ? block_sum_fixed(kin, wsum) : 0.0;
    unsigned *part = reinterpret_cast<unsigned *>(dv.partials);   // one word per block
    if (threadIdx.x == 0) {
        unsigned b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = max(b, wmax[w]);
        part[blockIdx.x] = b;
        if (nvt) dv.partials[(size_t)dv.maxblocks + blockIdx.x] = kblk;
        if (rule == 1) part[(size_t)6 * dv.maxblocks + blockIdx.x] = (unsigned)blk_half;
        __threadfence();
        const unsigned t = atomicAdd(&dv.flags->counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    unsigned b = 0;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x) b = max(b, __ldcg(part + k));
    b = __reduce_max_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = b;
    __syncthreads();
    if (nvt) {
        double k2 = 0.0;
        for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x)
            k2 += __ldcg(dv.partials + (size_t)dv.maxblocks + k);
        k2 = block_sum_fixed(k2, wsum);
        if (threadIdx.x == 0) {
            const double T = k2 / ((double)dv.d * (double)(dv.N - 1));
            dv.flags->nvt_T = T;
            dv.flags->nvt_lambda = T > 0.0 ? sqrt(fmax(0.0, 1.0 + rate * (T_target / T - 1.0))) : 1.0;
        }
    }
    if (rule == 1) {
        unsigned h = 0;
        for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x)
            h += __ldcg(part + (size_t)6 * dv.maxblocks + k);
        h = __reduce_add_sync(0xffffffffu, h);
        if ((threadIdx.x & 31) == 0) whalf[threadIdx.x >> 5] = h;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        unsigned m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, wmax[w]);
        unsigned half = 0;
        if (rule == 1)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) half += whalf[w];
        const float d2 = __uint_as_float(m);
        const float s2 = (float)(dv.skin * dv.skin) * (1.0f - 1e-5f);
        const bool finite = d2 <= 3.0e38f;
        int trig = (4.0f * d2 > s2) || !finite;
        if (rule == 1) {
            const long long st = ++dv.flags->md_step;
            trig = !finite || (st % n_bet == 0 &&
                               ((double)half >= 0.001 * (double)dv.N || d2 >= (float)(dv.skin * dv.skin)));
        }
        if (!finite || 16.0 * (double)d2 > dv.L * dv.L) atomicOr(&dv.flags->error, (int)ERR_LOST);
        dv.flags->rebuild = trig;
        if (cond) cudaGraphSetConditional(cond, trig ? 1u : 0u);
        dv.flags->counter = 0u;
    }
}

// pair forces of atom i with the list form of the system: packed entries
// (FP32 pair path only; the FP64 path takes the index bits alone)
template <int D, bool FP64P, typename FT, int LAW>
__device__ __forceinline__ void pair_forces_of(const Dev &dv, int i, int g, int lgG, int in_buf,
                                               FT (&f)[D], FT &e, FT &w, const uint32_t *stab) {
    if constexpr (FP64P || D > kMaxPackD) {
        pair_forces<D, FP64P, FT, LAW, false>(dv, i, g, lgG, in_buf, f, e, w);
    } else {
        if (dv.pack_sh) pair_forces<D, false, FT, LAW, true>(dv, i, g, lgG, in_buf, f, e, w, stab);
        else pair_forces<D, false, FT, LAW, false>(dv, i, g, lgG, in_buf, f, e, w);
    }
}

// The MD / force kernel.  Phase A: G lanes per atom accumulate the pair
// forces over the list and meet through xor shuffles; lane 0 parks the force
// in shared memory.  Phase B: the block's (atom, axis) items are spread over
// all threads, so the FP64 kick/drift arithmetic (the slow pipe on this GPU)
// runs with every lane busy and every SoA access coalesced.  Phase C writes
// the new gather rows (contiguous for the block) and folds the trigger.
template <int D, bool FP64P>
__global__ void __launch_bounds__(NT, HDMD_STEP_MIN_BLOCKS) k_step(Dev dv, StepCfg cfg) {
    using FT = typename std::conditional<FP64P, double, float>::type;
    constexpr int RF = Rows<D>::RF, RD = Rows<D>::RD;
    __shared__ double sh[(NT / 32) * kNRed];
    __shared__ FT sF[NT * D];
    __shared__ FT sE[NT], sW[NT];
    __shared__ float sDl[NT * D];   // (float) dlt of the drift, summed per atom in axis order
    __shared__ float sPos[FP64P ? 1 : NT * RF];
    __shared__ int sBad;
    // offset codes by stencil position, for packed list entries
    __shared__ uint32_t sStab[(!FP64P && D <= kMaxPackD) ? pow3(D) : 1];
    if (cfg.fire_red && dv.flags->fire[FS_STATUS] != (double)FIRE_RUNNING) return;  // loop ended
    if (!FP64P && D <= kMaxPackD && dv.pack_sh && cfg.compute_force) {
        for (int t = threadIdx.x; t < pow3(D); t += NT) sStab[t] = stencil_to_code<D>((uint32_t)t);
        __syncthreads();
    }
    const int G = dv.G, lgG = dv.lgG, APB = NT >> lgG;
    const int lgAPB = __ffs(NT) - 1 - lgG;   // APB is a power of two
    const int al = threadIdx.x >> lgG, g = threadIdx.x & (G - 1);
    const int base = blockIdx.x * APB;
    const int i = base + al;
    const bool valid = i < dv.N;
    const int Np = dv.Npad;
    if (threadIdx.x == 0) sBad = 0;

    if (cfg.compute_force) {
        FT f[D];
#pragma unroll
        for (int k = 0; k < D; ++k) f[k] = 0;
        FT e = 0, w = 0;
        if (valid) {
            if (dv.law == 1) pair_forces_of<D, FP64P, FT, 1>(dv, i, g, lgG, cfg.in_buf, f, e, w, sStab);
            else if (dv.law == 2) pair_forces_of<D, FP64P, FT, 2>(dv, i, g, lgG, cfg.in_buf, f, e, w, sStab);
            else pair_forces_of<D, FP64P, FT, 0>(dv, i, g, lgG, cfg.in_buf, f, e, w, sStab);
        }
        for (int o = G >> 1; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < D; ++k) f[k] += __shfl_xor_sync(0xffffffffu, f[k], o);
            e += __shfl_xor_sync(0xffffffffu, e, o);
            w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        if (g == 0) {
#pragma unroll
            for (int k = 0; k < D; ++k) sF[al * D + k] = f[k];
            sE[al] = e;
            sW[al] = w;
        }
    }
    __syncthreads();

    // ---- phase B: (axis, atom) items
    double acc[kNRed];
#pragma unroll
    for (int r = 0; r < kNRed; ++r) acc[r] = 0.0;
    const bool merged = cfg.kick2 && cfg.kick1_drift;
    const double kick = merged ? cfg.dt : cfg.halfdt;
    const bool do_kick = cfg.kick2 || cfg.kick1_drift;
    // Berendsen NVT: the second kick ends in v *= lambda (the paper fuses the
    // thermostat into it); sum m v^2 of those velocities feeds the next lambda
    const bool nvt = cfg.nvt && cfg.kick2;
    const double lam = nvt ? dv.flags->nvt_lambda : 1.0;
    double kin = 0.0;
    for (int t = threadIdx.x; t < APB * D; t += NT) {
        const int k = t >> lgAPB, a = t & (APB - 1), ii = base + a;
        if (ii >= dv.N) continue;
        const size_t o = (size_t)k * Np + ii;
        // v and dlt are read and written once per step: streaming accesses
        // (evict first), which leave L2 to the neighbour rows
        const double F = cfg.compute_force ? to_f64(sF[a * D + k]) : dv.F[o];
        if (cfg.store_F) dv.F[o] = F;
        const double im = dv.inv_mass ? dv.inv_mass[ii] : 1.0;
        double Fm = F;
        if (dv.inv_mass) Fm = F * im;   // a branch: no multiply without masses
        double v = HDMD_LDS(dv.v + o);
        if (nvt) {
            const double vf = (v + cfg.halfdt * Fm) * lam;
            kin += vf * vf / im;
            v = cfg.kick1_drift ? vf + cfg.halfdt * Fm : vf;
        } else if (do_kick) {
            v += kick * Fm;
        }
        if (cfg.thermo) acc[R_K2] += v * v / im;
        if (cfg.fire_red) {
            acc[R_P] += F * v;
            acc[R_VV] += v * v;
            acc[R_VF] += v * Fm;
            acc[R_FF] += Fm * Fm;
            acc[R_FN] += F * F;
        }
        if (cfg.kick1_drift) {
            const double dl = HDMD_LDS(dv.dlt + o) + cfg.dt * v;
            HDMD_STS(dv.dlt + o, dl);
            const float fl = to_f32(dl);
            sDl[a * D + k] = fl;
            if (FP64P) dv.gd[cfg.out_buf][(size_t)ii * RD + k] = dv.x0[o] + dl;
            else sPos[a * RF + k] = HDMD_LDS(dv.gs0 + (size_t)ii * RF + k) + fl;
        }
        if (do_kick) HDMD_STS(dv.v + o, v);
    }
    if (cfg.thermo || cfg.fire_red) {
        for (int a = threadIdx.x; a < APB; a += NT) {
            if (base + a >= dv.N) continue;
            acc[R_E] += (double)sE[a];
            acc[R_W] += (double)sW[a];
            if (cfg.fire_red) {
                double f2 = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) f2 += (double)sF[a * D + k] * (double)sF[a * D + k];
                acc[R_FMAX2] = fmax(acc[R_FMAX2], f2);
                if (!(f2 < INFINITY)) acc[R_BAD] = 1.0;
            }
        }
    }
    __syncthreads();

    // ---- phase C: rows out, trigger
    if (cfg.kick1_drift) {
        if (!FP64P) {
            float *go = dv.gs[cfg.out_buf];
            for (int t = threadIdx.x; t < APB * RF; t += NT) {
                const int a = t / RF, c = t - a * RF, ii = base + a;
                if (ii >= dv.N) continue;
                go[(size_t)ii * RF + c] = c < D ? sPos[a * RF + c] : HDMD_LDS(dv.gs0 + (size_t)ii * RF + c);
            }
        } else {
            for (int a = threadIdx.x; a < APB; a += NT)
                if (base + a < dv.N) dv.gd[cfg.out_buf][(size_t)(base + a) * RD + D] = 0.5 * dv.sigma[base + a];
        }
        unsigned mb = 0u;   // max of the float bits: a NaN orders above every number
        int half = 0;
        const float q2 = (float)(0.25 * dv.skin * dv.skin);
        for (int a = threadIdx.x; a < APB; a += NT) {
            if (base + a >= dv.N) continue;
            // |dlt|^2 of one atom, summed by one thread in axis order, so the
            // trigger (and the rebuild step it picks) repeats bit for bit
            float d2 = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) d2 = fmaf(sDl[a * D + k], sDl[a * D + k], d2);
            mb = max(mb, __float_as_uint(d2));
            half += d2 >= q2;
        }
        const int blk_half = cfg.rule == 1 ? __syncthreads_count(half) : 0;   // APB <= NT
        trigger_fold(dv, __uint_as_float(mb), false, cfg.cond_rebuild, nvt ? 1 : 0, kin, cfg.nvt_rate, cfg.nvt_T,
                     cfg.rule, cfg.n_bet, blk_half);
    }
    if (cfg.thermo || cfg.fire_red) {
        const bool last = block_reduce_and_fold<NT>(dv, acc, R_BAD + 1, dv.maxblocks, sh);
        if (last && threadIdx.x == 0 && cfg.fire_red) {
            const double *red = dv.red;
            // FIRE 2.0 scalar update (Guenole et al. 2020), one thread
            double *fs = dv.flags->fire;
            const int status = fire_scalar_update(fs, red);
            if (cfg.cond_loop) cudaGraphSetConditional(cfg.cond_loop, status == FIRE_RUNNING ? 1u : 0u);
        }
    }
}

// FIRE per-atom update, from the scalars the last force reduction left:
//   P <= 0 branch: x -= dt v / 2, v = 0;
//   then on both branches v += dt F/m; v = (1-alpha) v + alpha |v| F/|F|;
//   x += dt v.
// Block = NT/4 atoms; (axis, atom) items over all threads as in k_step.
template <int D>
__global__ void __launch_bounds__(NT) k_fire_update(Dev dv, int write_fp64_rows,
                                                    unsigned long long cond_rebuild) {
    constexpr int RF = Rows<D>::RF, RD = Rows<D>::RD;
    constexpr int APB = NT / 4;
    __shared__ float sPos[APB * RF];
    __shared__ float sDl[APB * D];
    __shared__ double sBack[APB * D], sStep[APB * D], sCB[APB], sCS[APB];
    const double *fs = dv.flags->fire;
    if (fs[FS_STATUS] != (double)FIRE_RUNNING) return;
    const double dt = fs[FS_DT], alpha = fs[FS_ALPHA];
    const bool up = fs[FS_BRANCH] != 0.0;
    const double vn = fs[FS_VNORM], fn = fs[FS_FNORM];
    const bool mix = fn > 0.0;
    const double cf = mix ? alpha * vn / fn : 0.0;
    const double dxm = fs[FP_DXMAX];
    const int base = blockIdx.x * APB;
    const int Np = dv.Npad;
    if (dxm > 0.0) {
        // Table II's displacement cap: an atom whose back-off (dt/2) v or
        // step dt v is longer than dx_max moves dx_max along it; the
        // per-atom lengths are summed over the axes in order (repeatable)
        for (int t = threadIdx.x; t < APB * D; t += NT) {
            const int k = t / APB, a = t - k * APB, ii = base + a;
            if (ii >= dv.N) continue;
            const size_t o = (size_t)k * Np + ii;
            const double im = dv.inv_mass ? dv.inv_mass[ii] : 1.0;
            double v = dv.v[o];
            const double F = dv.F[o];
            sBack[a * D + k] = up ? 0.0 : 0.5 * dt * v;
            if (!up) v = 0.0;
            v += dt * F * im;
            if (mix) v = (1.0 - alpha) * v + cf * F;
            dv.v[o] = v;
            sStep[a * D + k] = dt * v;
        }
        __syncthreads();
        for (int a = threadIdx.x; a < APB; a += NT) {
            double b2 = 0.0, s2 = 0.0;
            for (int k = 0; k < D; ++k) {
                b2 += sBack[a * D + k] * sBack[a * D + k];
                s2 += sStep[a * D + k] * sStep[a * D + k];
            }
            sCB[a] = b2 > dxm * dxm ? dxm / sqrt(b2) : 1.0;
            sCS[a] = s2 > dxm * dxm ? dxm / sqrt(s2) : 1.0;
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < APB * D; t += NT) {
        const int k = t / APB, a = t - k * APB, ii = base + a;
        if (ii >= dv.N) continue;
        const size_t o = (size_t)k * Np + ii;
        double dl = dv.dlt[o];
        if (dxm > 0.0) {
            dl -= sCB[a] * sBack[a * D + k];
            dl += sCS[a] * sStep[a * D + k];
        } else {
            const double im = dv.inv_mass ? dv.inv_mass[ii] : 1.0;
            double v = dv.v[o];
            const double F = dv.F[o];
            if (!up) {
                dl -= 0.5 * dt * v;
                v = 0.0;
            }
            v += dt * F * im;
            if (mix) v = (1.0 - alpha) * v + cf * F;
            dl += dt * v;
            dv.v[o] = v;
        }
        dv.dlt[o] = dl;
        const float fl = (float)dl;
        sDl[a * D + k] = fl;
        sPos[a * RF + k] = dv.gs0[(size_t)ii * RF + k] + fl;
        if (write_fp64_rows) dv.gd[0][(size_t)ii * RD + k] = dv.x0[o] + dl;
    }
    __syncthreads();
    float *go = dv.gs[0];
    for (int t = threadIdx.x; t < APB * RF; t += NT) {
        const int a = t / RF, c = t - a * RF, ii = base + a;
        if (ii >= dv.N) continue;
        go[(size_t)ii * RF + c] = c < D ? sPos[a * RF + c] : dv.gs0[(size_t)ii * RF + c];
    }
    if (write_fp64_rows)
        for (int a = threadIdx.x; a < APB; a += NT)
            if (base + a < dv.N) dv.gd[0][(size_t)(base + a) * RD + D] = 0.5 * dv.sigma[base + a];
    unsigned mb = 0u;   // max of the float bits: a NaN orders above every number
    for (int a = threadIdx.x; a < APB; a += NT) {
        if (base + a >= dv.N) continue;
        float d2 = 0.f;   // one thread per atom, axis order: repeatable
#pragma unroll
        for (int k = 0; k < D; ++k) d2 = fmaf(sDl[a * D + k], sDl[a * D + k], d2);
        mb = max(mb, __float_as_uint(d2));
    }
    trigger_fold(dv, __uint_as_float(mb), false, cond_rebuild);
}

// write gather rows of buffer buf from x0 + dlt (FP32 and/or FP64 rows)
template <int D>
__global__ void k_rows(Dev dv, int buf, int want32, int want64) {
    constexpr int RF = Rows<D>::RF, RD = Rows<D>::RD;
    const int i = blockIdx.x * NT + threadIdx.x;
    if (i >= dv.N) return;
    float *go = dv.gs[buf] + (size_t)i * RF;
    const float *g0 = dv.gs0 + (size_t)i * RF;
    double *gdo = dv.gd[buf] + (size_t)i * RD;
    for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * dv.Npad + i;
        const double dl = dv.dlt[o];
        if (want32) go[k] = g0[k] + (float)dl;
        if (want64) gdo[k] = dv.x0[o] + dl;
    }
    if (want32) go[D] = g0[D];
    if (want64) gdo[D] = 0.5 * dv.sigma[i];
}

template <int D>
void rows_impl(const Dev &dv, int buf, int w32, int w64, cudaStream_t s) {
    k_rows<D><<<(dv.N + NT - 1) / NT, NT, 0, s>>>(dv, buf, w32, w64);
}

template <int D>
void step_impl(const Dev &dv, const StepCfg &cfg, cudaStream_t s) {
    const int G = cfg.compute_force ? dv.G : 1;
    Dev d2 = dv;
    d2.G = G;   // without a force loop the lanes of a group have nothing to share
    d2.lgG = cfg.compute_force ? dv.lgG : 0;
    const int apb = NT / G;
    const int blocks = (dv.N + apb - 1) / apb;
    if (cfg.fp64_pairs)
        k_step<D, true><<<blocks, NT, 0, s>>>(cfg.compute_force ? dv : d2, cfg);
    else
        k_step<D, false><<<blocks, NT, 0, s>>>(cfg.compute_force ? dv : d2, cfg);
}

template <int D>
void fire_update_impl(const Dev &dv, int w64, unsigned long long cond, cudaStream_t s) {
    k_fire_update<D><<<(dv.N + NT / 4 - 1) / (NT / 4), NT, 0, s>>>(dv, w64, cond);
}

}  // namespace

void launch_step(const Dev &dv, const StepCfg &cfg, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, step_impl, dv, cfg, s);
}

void launch_rows(const Dev &dv, int buf, int want32, int want64, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, rows_impl, dv, buf, want32, want64, s);
}

void launch_fire_update(const Dev &dv, int write_fp64_rows, unsigned long long cond_rebuild,
                        cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, fire_update_impl, dv, write_fp64_rows, cond_rebuild, s);
}

}  // namespace hdmd
