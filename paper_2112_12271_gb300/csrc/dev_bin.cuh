// dev_bin.cuh -- per-item device functions of the cell binning (wrap,
// subcell index of Eq. (9), counting sort, reorder); kernels_bin.cu runs them
// one thread per item over the grid, the batched kernel over one block.
#pragma once
#include "common.cuh"

namespace hdmd {

__device__ __forceinline__ double wrap_box(double x, const Dev &dv, int &k) {
    double t = floor((x + dv.halfL) * dv.invL);
    x -= t * dv.L;
    k = (int)t;
    if (x >= dv.halfL) { x -= dv.L; k += 1; }
    if (x < -dv.halfL) { x += dv.L; k -= 1; }
    return x;
}

// atom i (old order): wrap, subcell index (axis 1 most significant), histogram;
// the per-atom state is copied aside for the reorder
template <int D>
__device__ __forceinline__ void assign_one(const Dev &dv, int i) {
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
        cell = cell * dv.n + ck;
    }
    dv.cell_of[i] = cell;
    dv.tsig[i] = dv.sigma[i];
    if (dv.inv_mass) dv.tim[i] = dv.inv_mass[i];
    dv.tid[i] = dv.id[i];
    atomicAdd(&dv.cell_count[cell], 1);
}

// exclusive scans of the histogram (-> cell_start) and of the home batches per
// cell (-> batch_start) by one block of 1024 threads or fewer (blockDim a
// multiple of 32); counters zeroed for the next build
__device__ __forceinline__ void scan_cells(const Dev &dv) {
    __shared__ int warp_sums[2][32];
    __shared__ int carry[2];
    const int H = home_batch(dv.d);
    const int NTs = blockDim.x;
    if (threadIdx.x < 2) carry[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = NTs >> 5;
    for (int base = 0; base < dv.ncells; base += NTs) {
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
            int w = lane < nw ? warp_sums[warp][lane] : 0;
            int wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            if (lane < nw) warp_sums[warp][lane] = wi - w;   // exclusive warp offsets
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
        if (threadIdx.x == NTs - 1) { carry[0] = excl + v; carry[1] = exclb + vb; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dv.cell_start[dv.ncells] = carry[0];
        dv.batch_start[dv.ncells] = carry[1];
    }
}

// members of each subcell, in arrival order, into the scratch array cellid
// (which the reorder step overwrites with the subcells of the new slots)
__device__ __forceinline__ void scatter_one(const Dev &dv, int i) {
    int c = dv.cell_of[i];
    int slot = atomicAdd(&dv.cell_fill[c], 1);
    dv.cellid[dv.cell_start[c] + slot] = i;
}

// position p of the scattered members: the member's rank by caller id among
// the members of its subcell places it, so every subcell comes out ordered by
// caller id whatever order the atomics gave.  One thread per member; the
// members of a subcell read the same entries in step, so a large subcell
// (a single subcell holds every atom) costs its size squared over its size
// threads rather than a serial sort.
__device__ __forceinline__ void rank_one(const Dev &dv, int p) {
    const int o = dv.cellid[p];
    const int c = dv.cell_of[o];
    const int a = dv.cell_start[c], b = dv.cell_start[c + 1];
    const int key = dv.tid[o];
    int r = 0;
    for (int q = a; q < b; ++q) r += dv.tid[dv.cellid[q]] < key;
    dv.perm[a + r] = o;
}

// new slot s: gather the state into cell order and write the build-time rows
// (cell-relative FP32 for the list build and the FP32 force loop, absolute
// FP64 for the FP64 force loop) into gather buffer buf
template <int D>
__device__ __forceinline__ void reorder_one(const Dev &dv, int s, int buf) {
    constexpr int RF = Rows<D>::RF, RD = Rows<D>::RD;
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

}  // namespace hdmd
