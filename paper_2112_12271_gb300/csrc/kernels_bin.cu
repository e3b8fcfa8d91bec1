// kernels_bin.cu -- state import/export and the cell binning of a list
// build: wrap into the box, linked-subcell assignment (Sec. II.C, Eqs.
// (7)-(9)), counting sort into cell order, and the reorder that makes the
// atoms of one subcell contiguous in memory.
//
// The paper assigns atoms to subcells serially; here it is a parallel
// counting sort: histogram (atomics) -> exclusive scan -> scatter -> a
// per-cell sort by caller id, so the resulting order (and every later sum)
// does not depend on atomic timing.
#include "dev_bin.cuh"
#include "launch.h"

namespace hdmd {

void launch_nbr_build(const Dev &dv, bool guarded, cudaStream_t s);  // kernels_nbr.cu

namespace {

constexpr int NT = 256;

__device__ __forceinline__ bool skip(const Dev &dv, bool guarded) {
    return guarded && *((volatile int *)&dv.flags->rebuild) == 0;
}

template <int D>
__global__ void k_import(Dev dv, const double *__restrict__ x_rm, const double *__restrict__ v_rm,
                         const double *__restrict__ mass) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.Npad) return;
    const bool real = i < dv.N;
    for (int k = 0; k < D; ++k) {
        size_t o = (size_t)k * dv.Npad + i;
        dv.x0[o] = real ? x_rm[(size_t)i * D + k] : 0.0;
        dv.dlt[o] = 0.0;
        dv.v[o] = (real && v_rm) ? v_rm[(size_t)i * D + k] : 0.0;
        dv.F[o] = 0.0;
        dv.img[o] = 0;
    }
    if (dv.inv_mass) dv.inv_mass[i] = (real && mass) ? 1.0 / mass[i] : 1.0;
    dv.id[i] = i;
}

__global__ void k_import_sigma(Dev dv, const double *__restrict__ sig_callerorder) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.N) return;
    dv.sigma[i] = sig_callerorder[dv.id[i]];
}

template <int D>
__global__ void k_export(Dev dv, double *x_rm, int32_t *img_rm, double *v_rm, double *f_rm,
                         double *sig) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= dv.N) return;
    const int c = dv.id[s];
    for (int k = 0; k < D; ++k) {
        size_t o = (size_t)k * dv.Npad + s;
        int kk;
        double xw = wrap_box(dv.x0[o] + dv.dlt[o], dv, kk);
        if (x_rm) x_rm[(size_t)c * D + k] = xw;
        if (img_rm) img_rm[(size_t)c * D + k] = dv.img[o] + kk;
        if (v_rm) v_rm[(size_t)c * D + k] = dv.v[o];
        if (f_rm) f_rm[(size_t)c * D + k] = dv.F[o];
    }
    if (sig) sig[c] = dv.sigma[s];
}

// step 1: wrap, subcell index, histogram; copy the per-atom state aside
template <int D>
__global__ void k_assign(Dev dv, bool guarded) {
    if (skip(dv, guarded)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < dv.N) {
        assign_one<D>(dv, i);
        dv.nnbr[i] = 0;   // list counters of the half-stencil build (atomics)
    }
}

// step 2: exclusive scans (one block) of the histogram -> cell_start, and of
// the number of home batches per cell -> batch_start; zero the counters
__global__ void __launch_bounds__(1024) k_scan(Dev dv, bool guarded) {
    if (skip(dv, guarded)) return;
    scan_cells(dv);
}

// step 3: scatter into cell order (order inside a cell fixed by step 4)
__global__ void k_scatter(Dev dv, bool guarded) {
    if (skip(dv, guarded)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < dv.N) scatter_one(dv, i);
}

// step 4: place each cell's members in caller-id order
__global__ void k_cell_sort(Dev dv, bool guarded) {
    if (skip(dv, guarded)) return;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < dv.N) rank_one(dv, p);
}

// step 5: gather the state into cell order; build-time rows
template <int D>
__global__ void k_reorder(Dev dv, int buf, bool guarded) {
    if (skip(dv, guarded)) return;
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) {
        dv.flags->nbuilds += 1;
        dv.flags->total_entries = 0;
    }
    if (s < dv.N) reorder_one<D>(dv, s, buf);
}

// trigger only: 2 max|dlt| > skin -> flags->rebuild
template <int D>
__global__ void k_trigger(Dev dv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.N) return;
    double s2 = 0.0;
    for (int k = 0; k < D; ++k) {
        double d = dv.dlt[(size_t)k * dv.Npad + i];
        s2 += d * d;
    }
    if (!(4.0 * s2 <= dv.skin * dv.skin)) atomicExch(&dv.flags->rebuild, 1);
}

__global__ void k_list_export(Dev dv, int32_t *counts, int32_t *idx, const int64_t *offsets) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= dv.N) return;
    const int c = dv.id[s];
    const int n = dv.nnbr[s];
    if (counts) counts[c] = n;
    if (idx) {
        int64_t off = offsets[c];
        for (int m = 0; m < n; ++m) idx[off + m] = dv.id[(uint32_t)dv.nbr[list_pos(m, s, dv.Npad, dv.lgG)] & dv.idx_mask];
    }
}

inline int nblk(int n) { return (n + NT - 1) / NT; }

template <int D> void import_impl(const Dev &dv, const double *x, const double *v, const double *m, cudaStream_t s) {
    k_import<D><<<nblk(dv.Npad), NT, 0, s>>>(dv, x, v, m);
}
template <int D> void export_impl(const Dev &dv, double *x, int32_t *img, double *v, double *f, double *sig, cudaStream_t s) {
    k_export<D><<<nblk(dv.N), NT, 0, s>>>(dv, x, img, v, f, sig);
}
template <int D> void rebuild_impl(const Dev &dv, int buf, bool guarded, cudaStream_t s) {
    k_assign<D><<<nblk(dv.N), NT, 0, s>>>(dv, guarded);
    k_scan<<<1, 1024, 0, s>>>(dv, guarded);
    k_scatter<<<nblk(dv.N), NT, 0, s>>>(dv, guarded);
    k_cell_sort<<<nblk(dv.N), NT, 0, s>>>(dv, guarded);
    k_reorder<D><<<nblk(dv.N), NT, 0, s>>>(dv, buf, guarded);
}
template <int D> void trigger_impl(const Dev &dv, cudaStream_t s) {
    k_trigger<D><<<nblk(dv.N), NT, 0, s>>>(dv);
}

}  // namespace

void launch_import(const Dev &dv, const double *x, const double *v, const double *m, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, import_impl, dv, x, v, m, s);
}
void launch_import_sigma(const Dev &dv, const double *sig, cudaStream_t s) {
    k_import_sigma<<<nblk(dv.N), NT, 0, s>>>(dv, sig);
}
void launch_export(const Dev &dv, double *x, int32_t *img, double *v, double *f, double *sig,
                   cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, export_impl, dv, x, img, v, f, sig, s);
}
void launch_rebuild(const Dev &dv, int buf, bool guarded, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, rebuild_impl, dv, buf, guarded, s);
    launch_nbr_build(dv, guarded, s);
}
void launch_check_trigger(const Dev &dv, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, trigger_impl, dv, s);
}
void launch_list_export(const Dev &dv, int32_t *counts, int32_t *idx, const int64_t *offsets,
                        cudaStream_t s) {
    k_list_export<<<nblk(dv.N), NT, 0, s>>>(dv, counts, idx, offsets);
}

}  // namespace hdmd
