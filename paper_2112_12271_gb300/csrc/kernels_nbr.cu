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
//     so after the counting sort their atoms lie in up to three ranges, read
//     with coalesced loads, one candidate per lane;
//   - 32 rows are set up at once, one per lane (offsets, reach tests, the
//     ranges), then the warp walks the reachable ones;
//   - each home atom tests the distance from itself to the row's box and to
//     the row's lower and upper subcell; only home atoms that can reach the
//     row test its candidates, and a subcell no home atom reaches is skipped;
//   - each home atom's hits are compacted with __ballot_sync/__popc, so the
//     lists come out in the same order on every run;
//   - a pair is kept iff r^2 < (sigma_ij + s)^2.  The FP32 distance
//     (cell-relative coordinates, error ~1e-7; for n_cell >= 3 in the
//     expanded form |r_j|^2 + |x_h|^2 - 2 r_j . x_h, bound in dev_nbr.cuh)
//     decides unless r^2 lies in a guard band around the cutoff, where the
//     FP64 distance decides, so the lists equal those of an all-FP64 search.
// With n_cell = 2 the offsets -1 and +1 name the same subcell, so each
// subcell is visited once (offsets {0, +1}) and every pair takes the minimum
// image along the axes where the two subcells differ; the paper switches to
// an all-pairs search there, which this amounts to.  A box shorter than
// 2 (sigma_max + s) (but longer than 2 sigma_max, so that only one image of a
// pair can interact) has a single subcell: all pairs, minimum image per axis.
#include "dev_nbr.cuh"
#include "launch.h"

namespace hdmd {
namespace {

constexpr int NT = 128;   // threads per block: 4 warps, one home batch each

// resident blocks per SM the register budget is sized for: d <= 4 tests all
// home atoms of a batch at once in 64 registers at 8 blocks; higher d keeps
// 80 registers at 6 blocks (more would spill)
#ifndef HDMD_NBR_MIN_BLOCKS
#define HDMD_NBR_MIN_BLOCKS 6
#endif
#ifndef HDMD_NBR_MIN_BLOCKS_LO
#define HDMD_NBR_MIN_BLOCKS_LO 8
#endif
__host__ __device__ constexpr bool nbr_allh(int D) { return D <= 4; }

template <int D, bool WRAP>
__global__ void __launch_bounds__(NT, nbr_allh(D) ? HDMD_NBR_MIN_BLOCKS_LO : HDMD_NBR_MIN_BLOCKS)
k_nbr_build(Dev dv, bool guarded) {
    if (guarded && *((volatile int *)&dv.flags->rebuild) == 0) return;
    const int w = (blockIdx.x * NT + threadIdx.x) >> 5;
    if (w >= dv.batch_start[dv.ncells]) return;   // warp-uniform
    nbr_batch<D, WRAP, nbr_allh(D)>(dv, w, threadIdx.x & 31);
}

// n_cell >= 3: one warp per home subcell, its atoms staged in shared memory
// (nbr_cell)
#ifndef HDMD_NBR_CELL_MIN_BLOCKS
#define HDMD_NBR_CELL_MIN_BLOCKS 8
#endif
template <int D, bool HALF>
__global__ void __launch_bounds__(NT, HDMD_NBR_CELL_MIN_BLOCKS) k_nbr_cell(Dev dv, bool guarded) {
    __shared__ __align__(16) float sh[(NT / 32) * 32 * home_row_floats(D)];
    if (guarded && *((volatile int *)&dv.flags->rebuild) == 0) return;
    const int warp = threadIdx.x >> 5;
    const int c = blockIdx.x * (NT / 32) + warp;
    if (c >= dv.ncells) return;   // warp-uniform; no block barrier follows
    nbr_cell<D, HALF>(dv, c, threadIdx.x & 31, sh + warp * 32 * home_row_floats(D));
}

// After the half-stencil build: every list sorted by neighbour index (its
// entries arrived in the order of the atomics that placed them; the code word
// travels with its entry), the counts clamped to the capacity, and the
// longest list and the total number of entries reported (one atomic per
// block).  One warp per list: the lanes hold the entries (up to kFinishK per
// lane), each entry's rank is the number of smaller neighbour indices
// (distinct within a list) counted through shuffles, and every entry is
// written back at its rank; longer lists are sorted by one lane.
constexpr int kFinishK = 4;   // entries per lane: lists up to 128 sorted by the warp
__global__ void __launch_bounds__(NT) k_list_finish(Dev dv, bool guarded) {
    __shared__ int smax[NT / 32];
    __shared__ unsigned long long ssum[NT / 32];
    if (guarded && *((volatile int *)&dv.flags->rebuild) == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (NT / 32);
    const bool packed = dv.pack_sh > 0;
    const uint32_t msk = packed ? dv.idx_mask : 0xffffffffu;
    uint32_t *nb = reinterpret_cast<uint32_t *>(dv.nbr);
    int mx = 0;
    unsigned long long sm = 0;
    for (int i = blockIdx.x * (NT / 32) + warp; i < dv.N; i += nwarps) {
        const int raw = dv.nnbr[i];
        const int n = min(raw, dv.cap);
        mx = max(mx, raw);
        sm += (unsigned long long)raw;
        if (n <= 32 * kFinishK) {
            uint32_t e[kFinishK], cd[kFinishK], key[kFinishK];
#pragma unroll
            for (int q = 0; q < kFinishK; ++q) {
                const int m = q * 32 + lane;
                e[q] = 0u;
                cd[q] = 0u;
                key[q] = 0xffffffffu;
                if (m < n) {
                    const int64_t pm = list_pos(m, i, dv.Npad, dv.lgG);
                    e[q] = nb[pm];
                    if (!packed) cd[q] = dv.code[pm];
                    key[q] = e[q] & msk;
                }
            }
            int rank[kFinishK] = {};
#pragma unroll
            for (int q2 = 0; q2 < kFinishK; ++q2) {
                if (q2 * 32 >= n) break;
                const int cnt = min(32, n - q2 * 32);
                for (int l2 = 0; l2 < cnt; ++l2) {
                    const uint32_t k2 = __shfl_sync(0xffffffffu, key[q2], l2);
#pragma unroll
                    for (int q = 0; q < kFinishK; ++q) rank[q] += k2 < key[q];
                }
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < kFinishK; ++q) {
                if (q * 32 + lane < n) {
                    const int64_t pr = list_pos(rank[q], i, dv.Npad, dv.lgG);
                    nb[pr] = e[q];
                    if (!packed) dv.code[pr] = cd[q];
                }
            }
        } else if (lane == 0) {
            for (int m = 1; m < n; ++m) {   // insertion sort by one lane
                const int64_t pm = list_pos(m, i, dv.Npad, dv.lgG);
                const uint32_t e = nb[pm], key = e & msk;
                const uint32_t cd = packed ? 0u : dv.code[pm];
                int k = m - 1;
                for (; k >= 0; --k) {
                    const int64_t pk = list_pos(k, i, dv.Npad, dv.lgG);
                    const uint32_t ek = nb[pk];
                    if ((ek & msk) <= key) break;
                    const int64_t pk1 = list_pos(k + 1, i, dv.Npad, dv.lgG);
                    nb[pk1] = ek;
                    if (!packed) dv.code[pk1] = dv.code[pk];
                }
                const int64_t pk1 = list_pos(k + 1, i, dv.Npad, dv.lgG);
                nb[pk1] = e;
                if (!packed) dv.code[pk1] = cd;
            }
        }
        if (lane == 0) {
            dv.nnbr[i] = n;
            if (raw > dv.cap) atomicOr(&dv.flags->error, (int)ERR_OVERFLOW);
        }
        __syncwarp();
    }
    if (lane == 0) {
        smax[warp] = mx;
        ssum[warp] = sm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < NT / 32; ++w) {
            mx = max(mx, smax[w]);
            sm += ssum[w];
        }
        atomicMax(&dv.flags->max_count, mx);
        atomicAdd((unsigned long long *)&dv.flags->total_entries, sm);
    }
}

// The half-stencil build where a home atom has many candidates (3^d times
// the atoms per subcell): it tests each pair once but pays atomics for the
// slots and a sort of every list.  Build times on one GB300, half / full
// stencil: d=6 N=32768 (5832 candidates) 0.289 / 0.376 ms, N=2^21 (5832)
// 10.7 / 14.9 ms, the paper's model at N=10^5: d=6 (17.8k) 1.29 / 1.75 ms,
// d=5 (3.1k) 0.478 / 0.548 ms, d=4 (550) 0.249 / 0.217 ms, d=3 (100)
// 0.189 / 0.156 ms.
constexpr double kHalfStencilCandidates = 1500.0;
inline bool half_stencil(const Dev &dv, int stencil) {
    return (double)stencil * (double)dv.N >= kHalfStencilCandidates * (double)dv.ncells;
}

template <int D>
void nbr_impl(const Dev &dv, bool guarded, cudaStream_t s) {
    if (dv.n >= 3) {
        const int blocks = (dv.ncells + NT / 32 - 1) / (NT / 32);
        if (half_stencil(dv, pow3(D))) {
            k_nbr_cell<D, true><<<blocks, NT, 0, s>>>(dv, guarded);
            const int warps = (dv.N + 0) < 152 * 8 * (NT / 32) ? dv.N : 152 * 8 * (NT / 32);
            if (dv.N > 0) k_list_finish<<<(warps + NT / 32 - 1) / (NT / 32), NT, 0, s>>>(dv, guarded);
        } else {
            k_nbr_cell<D, false><<<blocks, NT, 0, s>>>(dv, guarded);
        }
        return;
    }
    // upper bound on the number of home batches: N / H + n_cells
    const int64_t warps = (int64_t)dv.N / home_batch(D) + dv.ncells + 1;
    const int blocks = (int)((warps * 32 + NT - 1) / NT);
    k_nbr_build<D, false><<<blocks, NT, 0, s>>>(dv, guarded);
}

}  // namespace

void launch_nbr_build(const Dev &dv, bool guarded, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, nbr_impl, dv, guarded, s);
}

}  // namespace hdmd
