// batch_impl.cuh -- many independent jobs (FIRE minimisations or MD runs of
// uneven N and d) in one persistent launch.
//
// One thread block owns one job at a time and runs the whole method on it:
// binning and Verlet lists (Sec. II.C), pair forces (Sec. II.B getforce),
// FIRE 2.0 or velocity Verlet (Sec. II.B), the displacement trigger.  All
// synchronisation of a job is __syncthreads inside its block, so the jobs
// need no grid-wide barrier; blocks take jobs from a queue (largest first,
// ordered by the host) until it is empty.  The per-atom device functions are
// those of the single-system kernels (dev_*.cuh), so the physics is the same
// code.  A launch runs each job for at most `budget` iterations or steps and
// saves its progress, so the host can refill finished slots between launches
// (the serving loop) or run everything to the end in one launch (budget 0).
// Reductions are block trees in a fixed order: a job gives the same bits
// whichever block runs it and whatever else is in the batch.
#pragma once
#include <type_traits>

#include "batch.cuh"
#include "dev_bin.cuh"
#include "dev_fire.cuh"
#include "dev_force.cuh"
#include "dev_nbr.cuh"
#include "launch.h"

namespace hdmd {
namespace {

// The block size is the launch's (kBatchNT, or kBatchWideNT for the jobs
// above kBatchWideN atoms): a job always runs in blocks of the same size, so
// its reductions, and its result, do not depend on the rest of the batch.
#define BT ((int)blockDim.x)
#define NWB ((int)(blockDim.x >> 5))
constexpr int kMaxWarpsB = 32;

__device__ __forceinline__ double blk_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < NWB; ++w) t += sh[w];
    return t;
}

__device__ __forceinline__ double blk_max(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < NWB; ++w) t = fmax(t, sh[w]);
    return t;
}

// full list build of one job by one block
template <int D>
__device__ bool blk_build(const Dev &dv) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < dv.N; i += BT) assign_one<D>(dv, i);
    __syncthreads();
    scan_cells(dv);
    __syncthreads();
    for (int i = tid; i < dv.N; i += BT) scatter_one(dv, i);
    __syncthreads();
    for (int p = tid; p < dv.N; p += BT) rank_one(dv, p);
    __syncthreads();
    for (int s = tid; s < dv.N; s += BT) reorder_one<D>(dv, s, 0);
    if (tid == 0) {
        dv.flags->nbuilds += 1;
        dv.flags->total_entries = 0;
    }
    __syncthreads();
    const int nb = dv.batch_start[dv.ncells];
    if (dv.n >= 3) {
        for (int w = warp; w < nb; w += NWB) nbr_batch<D, true>(dv, w, lane);
    } else {
        for (int w = warp; w < nb; w += NWB) nbr_batch<D, false>(dv, w, lane);
    }
    __syncthreads();
    return (*(volatile int *)&dv.flags->error & ERR_OVERFLOW) == 0;
}

// forces of all atoms into dv.F; sums of the energy/virial (thermo) or of the
// FIRE scalars into J.sums (Red slots)
template <int D, bool FP64P>
__device__ void blk_force(BatchJob &J, const Dev &dv, int lgG, bool fire, double *sh) {
    using FT = typename std::conditional<FP64P, double, float>::type;
    const int tid = threadIdx.x;
    const int G = 1 << lgG, APB = BT >> lgG;
    const int g = tid & (G - 1), al = tid >> lgG;
    const int Np = dv.Npad;
    double aE = 0, aW = 0, aP = 0, aVV = 0, aVF = 0, aFF = 0, aFN = 0, aMax = 0, aBad = 0;
    for (int base = 0; base < dv.N; base += APB) {
        const int i = base + al;
        FT f[D];
#pragma unroll
        for (int k = 0; k < D; ++k) f[k] = 0;
        FT e = 0, w = 0;
        if (i < dv.N) pair_forces<D, FP64P, FT, 0>(dv, i, g, lgG, 0, f, e, w);
        for (int o = G >> 1; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < D; ++k) f[k] += __shfl_xor_sync(0xffffffffu, f[k], o);
            e += __shfl_xor_sync(0xffffffffu, e, o);
            w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        if (g == 0 && i < dv.N) {
            const double im = dv.inv_mass ? dv.inv_mass[i] : 1.0;
            double f2 = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double F = (double)f[k];
                const size_t o = (size_t)k * Np + i;
                dv.F[o] = F;
                f2 += F * F;
                if (fire) {
                    const double v = dv.v[o], Fm = F * im;
                    aP += F * v;
                    aVV += v * v;
                    aVF += v * Fm;
                    aFF += Fm * Fm;
                    aFN += F * F;
                }
            }
            aE += (double)e;
            aW += (double)w;
            aMax = fmax(aMax, f2);
            if (!(f2 < INFINITY)) aBad = 1.0;
        }
    }
    const double sE = blk_sum(aE, sh), sW = blk_sum(aW, sh), sM = blk_max(aMax, sh);
    const double sB = blk_max(aBad, sh);
    double sP = 0, sVV = 0, sVF = 0, sFF = 0, sFN = 0;
    if (fire) {
        sP = blk_sum(aP, sh);
        sVV = blk_sum(aVV, sh);
        sVF = blk_sum(aVF, sh);
        sFF = blk_sum(aFF, sh);
        sFN = blk_sum(aFN, sh);
    }
    if (tid == 0) {
        J.sums[R_E] = sE;
        J.sums[R_W] = sW;
        J.sums[R_FMAX2] = sM;
        J.sums[R_BAD] = sB;
        J.sums[R_P] = sP;
        J.sums[R_VV] = sVV;
        J.sums[R_VF] = sVF;
        J.sums[R_FF] = sFF;
        J.sums[R_FN] = sFN;
    }
    __syncthreads();
}

template <int D>
__device__ void blk_force_any(BatchJob &J, const Dev &dv, bool fp64, int lgG, bool fire, double *sh) {
    if (fp64) blk_force<D, true>(J, dv, lgG, fire, sh);
    else blk_force<D, false>(J, dv, lgG, fire, sh);
}

// rows of the gather buffer from x0 + dlt, and the trigger: returns 0 (lists
// valid), 1 (rebuild) or 2 (lost atom: non-finite or beyond L/4); the value
// is the same in every thread
template <int D>
__device__ int blk_rows_trigger(BatchJob &J, const Dev &dv, bool write64, double *sh) {
    constexpr int RF = Rows<D>::RF, RD = Rows<D>::RD;
    double m = 0.0;
    for (int i = threadIdx.x; i < dv.N; i += BT) {
        float d2 = 0.f;
        float *go = dv.gs[0] + (size_t)i * RF;
        const float *g0 = dv.gs0 + (size_t)i * RF;
        double *gdo = dv.gd[0] + (size_t)i * RD;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const size_t o = (size_t)k * dv.Npad + i;
            const double dl = dv.dlt[o];
            const float fl = (float)dl;
            d2 = fmaf(fl, fl, d2);
            go[k] = g0[k] + fl;
            if (write64) gdo[k] = dv.x0[o] + dl;
        }
        go[D] = g0[D];
        if (write64) gdo[D] = 0.5 * dv.sigma[i];
        m = fmax(m, (double)(d2 <= 3.0e38f ? d2 : 3.0e38f));
        if (!(d2 <= 3.0e38f)) m = INFINITY;
    }
    const double mx = blk_max(m, sh);
    const bool finite = mx < INFINITY;
    if (!finite || 16.0 * mx > dv.L * dv.L) {
        if (threadIdx.x == 0) J.error |= ERR_LOST;
        return 2;
    }
    return 4.0 * mx > dv.skin * dv.skin * (1.0 - 1e-5) ? 1 : 0;
}

// FIRE per-atom update (same rule as the single-system kernel)
template <int D>
__device__ void blk_fire_update(BatchJob &J, const Dev &dv) {
    const double *fs = J.fire;
    const double dt = fs[FS_DT], alpha = fs[FS_ALPHA];
    const bool up = fs[FS_BRANCH] != 0.0;
    const double vn = fs[FS_VNORM], fn = fs[FS_FNORM];
    const bool mix = fn > 0.0;
    const double cf = mix ? alpha * vn / fn : 0.0;
    for (int k = 0; k < D; ++k) {
        for (int i = threadIdx.x; i < dv.N; i += BT) {
            const size_t o = (size_t)k * dv.Npad + i;
            const double im = dv.inv_mass ? dv.inv_mass[i] : 1.0;
            double v = dv.v[o], dl = dv.dlt[o];
            const double F = dv.F[o];
            if (!up) {
                dl -= 0.5 * dt * v;
                v = 0.0;
            }
            v += dt * F * im;
            if (mix) v = (1.0 - alpha) * v + cf * F;
            dl += dt * v;
            dv.v[o] = v;
            dv.dlt[o] = dl;
        }
    }
    __syncthreads();
}

// velocity Verlet half kick; with drift, then x += dt v
template <int D>
__device__ double blk_kick(const Dev &dv, double halfdt, double dt, bool drift, bool kinetic) {
    double K2 = 0.0;
    for (int k = 0; k < D; ++k) {
        for (int i = threadIdx.x; i < dv.N; i += BT) {
            const size_t o = (size_t)k * dv.Npad + i;
            const double im = dv.inv_mass ? dv.inv_mass[i] : 1.0;
            double v = dv.v[o] + halfdt * dv.F[o] * im;
            dv.v[o] = v;
            if (drift) dv.dlt[o] += dt * v;
            if (kinetic) K2 += v * v / im;
        }
    }
    __syncthreads();
    return K2;
}

template <int D>
__device__ void run_job(BatchJob &J, long long budget) {
    __shared__ Dev sdv;
    __shared__ double sh[kMaxWarpsB];
    __shared__ int s_st;
    if (threadIdx.x == 0) {
        sdv = J.dv;
        sdv.lgG = J.lgG;   // the list layout follows the job's lanes per atom
        sdv.G = 1 << J.lgG;
    }
    __syncthreads();
    const Dev &dv = sdv;
    if (J.status != JOB_ACTIVE) return;
    const int lgG = J.lgG;
    const bool fire = J.kind == JOB_FIRE;
    if (!J.built) {
        const bool ok = blk_build<D>(dv);
        if (threadIdx.x == 0) {
            J.built = 1;
            J.builds += 1;
            if (!ok) { J.error |= ERR_OVERFLOW; J.status = JOB_ERROR; }
        }
        __syncthreads();
        if (!ok) return;
    }
    if (!J.force_valid) {
        blk_force_any<D>(J, dv, J.phase64 != 0, lgG, fire, sh);
        if (threadIdx.x == 0) J.force_valid = 1;
        __syncthreads();
    }
    long long it = 0;
    while (budget == 0 || it < budget) {
        if (fire) {
            if (threadIdx.x == 0) s_st = fire_scalar_update(J.fire, J.sums);
            __syncthreads();
            const int st = s_st;
            if (st == FIRE_SWITCH) {
                // the same iteration continues with FP64 pair forces
                if (threadIdx.x == 0) {
                    J.fire[FP_SWITCH] = 0.0;
                    J.fire[FS_STATUS] = FIRE_RUNNING;
                    J.fire[FS_PHASE_ITER] = 0.0;
                    J.fire[FS_NNEG] = 0.0;
                    J.fire[FS_NPOS] = 0.0;
                    J.phase64 = 1;
                }
                __syncthreads();
                blk_rows_trigger<D>(J, dv, true, sh);
                blk_force_any<D>(J, dv, true, lgG, true, sh);
                continue;
            }
            if (st != FIRE_RUNNING) {
                if (threadIdx.x == 0) J.status = st == FIRE_CONVERGED ? JOB_DONE : JOB_NOT_CONVERGED;
                break;
            }
            blk_fire_update<D>(J, dv);
        } else {
            if (J.steps_done >= J.nsteps) {
                if (threadIdx.x == 0) J.status = JOB_DONE;
                break;
            }
            blk_kick<D>(dv, 0.5 * J.dt, J.dt, true, false);
        }
        const bool p64 = J.phase64 != 0;
        const int trig = blk_rows_trigger<D>(J, dv, p64, sh);
        if (trig == 2) {
            if (threadIdx.x == 0) J.status = JOB_ERROR;
            break;
        }
        if (trig == 1) {
            const bool ok = blk_build<D>(dv);
            if (threadIdx.x == 0) {
                J.builds += 1;
                if (!ok) { J.error |= ERR_OVERFLOW; J.status = JOB_ERROR; }
            }
            __syncthreads();
            if (!ok) break;
        }
        blk_force_any<D>(J, dv, p64, lgG, fire, sh);
        if (!fire) {
            const bool last = J.steps_done + 1 >= J.nsteps;
            const double K2 = blk_kick<D>(dv, 0.5 * J.dt, J.dt, false, last);
            if (last) {
                const double k2 = blk_sum(K2, sh);
                if (threadIdx.x == 0) J.sums[R_K2] = k2;
            }
            if (threadIdx.x == 0) J.steps_done += 1;
        }
        __syncthreads();
        ++it;
    }
    __syncthreads();
}

template <int D>
__device__ __forceinline__ void batch_queue(BatchJob *jobs, const int *order, BatchCtl *ctl) {
    __shared__ int s_q;
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(&ctl->next, 1);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        if (q >= ctl->njobs) return;
        run_job<D>(jobs[order[ctl->first + q]], ctl->budget);
    }
}

template <int D>
__global__ void __launch_bounds__(kBatchNT, 2) k_batch(BatchJob *jobs, const int *order, BatchCtl *ctl) {
    batch_queue<D>(jobs, order, ctl);
}

template <int D>
__global__ void __launch_bounds__(kBatchWideNT, 1) k_batch_wide(BatchJob *jobs, const int *order,
                                                               BatchCtl *ctl) {
    batch_queue<D>(jobs, order, ctl);
}

template <int D>
__global__ void __launch_bounds__(kBatchNT, 2) k_batch_probe(BatchJob *job, int reps) {
    __shared__ Dev sdv;
    __shared__ double sh[kMaxWarpsB];
    BatchJob &J = *job;
    if (threadIdx.x == 0) {
        sdv = J.dv;
        sdv.lgG = J.lgG;
        sdv.G = 1 << J.lgG;
    }
    __syncthreads();
    const Dev &dv = sdv;
    if (!J.built) {
        const bool ok = blk_build<D>(dv);
        if (threadIdx.x == 0) {
            J.built = 1;
            J.builds += 1;
            if (!ok) { J.error |= ERR_OVERFLOW; J.status = JOB_ERROR; }
        }
        __syncthreads();
        if (!ok) return;
    }
    for (int r = 0; r < reps; ++r) blk_force_any<D>(J, dv, J.phase64 != 0, J.lgG, J.kind == JOB_FIRE, sh);
    if (threadIdx.x == 0) J.force_valid = 1;
}

}  // namespace

// the including translation unit instantiates the launchers of its dimensions
#define HDMD_BATCH_INSTANTIATE(D)                                                      \
    void launch_batch_d##D(BatchJob *jobs, const int *order, BatchCtl *ctl, int grid,  \
                           cudaStream_t s) {                                           \
        k_batch<D><<<grid, kBatchNT, 0, s>>>(jobs, order, ctl);                        \
    }                                                                                  \
    void launch_batch_wide_d##D(BatchJob *jobs, const int *order, BatchCtl *ctl,       \
                                int grid, cudaStream_t s) {                            \
        k_batch_wide<D><<<grid, kBatchWideNT, 0, s>>>(jobs, order, ctl);               \
    }                                                                                  \
    void launch_batch_probe_d##D(BatchJob *job, int reps, cudaStream_t s) {            \
        k_batch_probe<D><<<1, kBatchNT, 0, s>>>(job, reps);                            \
    }

}  // namespace hdmd
#undef BT
#undef NWB
