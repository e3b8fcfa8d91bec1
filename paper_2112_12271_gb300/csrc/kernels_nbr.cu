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
template <int D>
__global__ void __launch_bounds__(NT, HDMD_NBR_CELL_MIN_BLOCKS) k_nbr_cell(Dev dv, bool guarded) {
    __shared__ __align__(16) float sh[(NT / 32) * 32 * home_row_floats(D)];
    if (guarded && *((volatile int *)&dv.flags->rebuild) == 0) return;
    const int warp = threadIdx.x >> 5;
    const int c = blockIdx.x * (NT / 32) + warp;
    if (c >= dv.ncells) return;   // warp-uniform; no block barrier follows
    nbr_cell<D>(dv, c, threadIdx.x & 31, sh + warp * 32 * home_row_floats(D));
}

template <int D>
void nbr_impl(const Dev &dv, bool guarded, cudaStream_t s) {
    if (dv.n >= 3) {
        const int blocks = (dv.ncells + NT / 32 - 1) / (NT / 32);
        k_nbr_cell<D><<<blocks, NT, 0, s>>>(dv, guarded);
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
