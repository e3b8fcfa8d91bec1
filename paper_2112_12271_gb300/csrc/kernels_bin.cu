// kernels_bin.cu -- state import/export and the cell binning of a list
// build: wrap into the box, linked-subcell assignment (Sec. II.C, Eqs.
// (7)-(9)), counting sort into cell order, and the reorder that makes the
// atoms of one subcell contiguous in memory.
//
// The paper assigns atoms to subcells serially; here it is a parallel
// counting sort: histogram (atomics) -> exclusive scan -> scatter -> a
// per-cell sort by caller id, so the resulting order (and every later sum)
// does not depend on atomic timing.
#include "launch.h"

namespace hdmd {

void launch_nbr_build(const Dev &dv, bool guarded, cudaStream_t s);  // kernels_nbr.cu

namespace {

constexpr int NT = 256;

__device__ __forceinline__ bool skip(const Dev &dv, bool guarded) {
    return guarded && *((volatile int *)&dv.flags->rebuild) == 0;
}

// wrap a coordinate into [-L/2, L/2); returns the number of box lengths removed
__device__ __forceinline__ double wrap_box(double x, const Dev &dv, int &k) {
    double t = floor((x + dv.halfL) * dv.invL);
    x -= t * dv.L;
    k = (int)t;
    if (x >= dv.halfL) { x -= dv.L; k += 1; }
    if (x < -dv.halfL) { x += dv.L; k -= 1; }
    return x;
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
    if (i >= dv.N) return;
    int cell = 0;
    for (int k = 0; k < D; ++k) {
        size_t o = (size_t)k * dv.Npad + i;
        int kk;
        double xw = wrap_box(dv.x0[o] + dv.dlt[o], dv, kk);
        dv.tx[o] = xw;
        dv.timg[o] = dv.img[o] + kk;
        dv.tv[o] = dv.v[o];
        int ck = (int)floor((xw + dv.halfL) * dv.invLsc);
        ck = ck < 0 ? 0 : (ck > dv.n - 1 ? dv.n - 1 : ck);   // round-off at the upper face
        cell = cell * dv.n + ck;                              // Eq. (9), axis 1 most significant
    }
    dv.cell_of[i] = cell;
    dv.tsig[i] = dv.sigma[i];
    if (dv.inv_mass) dv.tim[i] = dv.inv_mass[i];
    dv.tid[i] = dv.id[i];
    atomicAdd(&dv.cell_count[cell], 1);
}

// step 2: exclusive scans (one block) of the histogram -> cell_start, and of
// the number of home batches per cell -> batch_start; zero the counters
__global__ void __launch_bounds__(1024) k_scan(Dev dv, bool guarded) {
    if (skip(dv, guarded)) return;
    __shared__ int warp_sums[2][32];
    __shared__ int carry[2];
    const int H = home_batch(dv.d);
    if (threadIdx.x < 2) carry[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < dv.ncells; base += 1024) {
        const int c = base + threadIdx.x;
        const int v = c < dv.ncells ? dv.cell_count[c] : 0;
        const int vb = (v + H - 1) / H;
        int incl = v, inclb = vb;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            int tb = __shfl_up_sync(0xffffffffu, inclb, o);
            if (lane >= o) { incl += t; inclb += tb; }
        }
        if (lane == 31) { warp_sums[0][warp] = incl; warp_sums[1][warp] = inclb; }
        __syncthreads();
        if (warp < 2) {
            int w = warp_sums[warp][lane];
            int wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            warp_sums[warp][lane] = wi - w;   // exclusive warp offsets
        }
        __syncthreads();
        const int excl = carry[0] + warp_sums[0][warp] + incl - v;
        const int exclb = carry[1] + warp_sums[1][warp] + inclb - vb;
        if (c < dv.ncells) {
            dv.cell_start[c] = excl;
            dv.batch_start[c] = exclb;
            dv.cell_fill[c] = 0;
            dv.cell_count[c] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 1023) { carry[0] = excl + v; carry[1] = exclb + vb; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dv.cell_start[dv.ncells] = carry[0];
        dv.batch_start[dv.ncells] = carry[1];
    }
}

// step 3: scatter into cell order (order inside a cell fixed by step 4)
__global__ void k_scatter(Dev dv, bool guarded) {
    if (skip(dv, guarded)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.N) return;
    int c = dv.cell_of[i];
    int slot = atomicAdd(&dv.cell_fill[c], 1);
    dv.perm[dv.cell_start[c] + slot] = i;
}

// step 4: sort each cell's members by caller id (insertion sort; cells are small)
__global__ void k_cell_sort(Dev dv, bool guarded) {
    if (skip(dv, guarded)) return;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= dv.ncells) return;
    int a = dv.cell_start[c], b = dv.cell_start[c + 1];
    for (int p = a + 1; p < b; ++p) {
        int v = dv.perm[p];
        int key = dv.tid[v];
        int q = p - 1;
        while (q >= a && dv.tid[dv.perm[q]] > key) {
            dv.perm[q + 1] = dv.perm[q];
            --q;
        }
        dv.perm[q + 1] = v;
    }
}

// step 5: gather the state into cell order; build-time rows for the list
// build (cell-relative FP32) and for both force loops
template <int D>
__global__ void k_reorder(Dev dv, int buf, bool guarded) {
    if (skip(dv, guarded)) return;
    constexpr int RF = Rows<D>::RF, RD = Rows<D>::RD;
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) {
        dv.flags->nbuilds += 1;
        dv.flags->total_entries = 0;
    }
    if (s >= dv.N) return;
    const int o = dv.perm[s];
    int cell = dv.cell_of[o];
    dv.cellid[s] = cell;
    int C[D];
    for (int k = D - 1; k >= 0; --k) { C[k] = cell % dv.n; cell /= dv.n; }
    const double sg = dv.tsig[o];
    const float half_sg = (float)(0.5 * sg);
    float *r0 = dv.gs0 + (size_t)s * RF;
    float *r1 = dv.gs[buf] + (size_t)s * RF;
    double *rd = dv.gd[buf] + (size_t)s * RD;
    for (int k = 0; k < D; ++k) {
        size_t so = (size_t)k * dv.Npad + s, oo = (size_t)k * dv.Npad + o;
        double x = dv.tx[oo];
        dv.x0[so] = x;
        dv.dlt[so] = 0.0;
        dv.v[so] = dv.tv[oo];
        dv.img[so] = dv.timg[oo];
        double centre = -dv.halfL + (C[k] + 0.5) * dv.Lsc;     // Eq. (8)
        float rel = (float)(x - centre);
        r0[k] = rel;
        r1[k] = rel;
        rd[k] = x;
    }
    r0[D] = half_sg;
    r1[D] = half_sg;
    rd[D] = 0.5 * sg;
    for (int k = D + 1; k < RF; ++k) { r0[k] = 0.f; r1[k] = 0.f; }
    for (int k = D + 1; k < RD; ++k) rd[k] = 0.0;
    dv.sigma[s] = sg;
    if (dv.inv_mass) dv.inv_mass[s] = dv.tim[o];
    dv.id[s] = dv.tid[o];
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
        for (int m = 0; m < n; ++m) idx[off + m] = dv.id[dv.nbr[list_pos(m, s, dv.Npad, dv.lgG)]];
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
    k_cell_sort<<<nblk(dv.ncells), NT, 0, s>>>(dv, guarded);
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
