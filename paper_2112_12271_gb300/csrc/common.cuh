// common.cuh -- device-side data layout shared by the kernels of the hdmd
// library (d-dimensional soft-sphere MD, arXiv:2112.12271).
//
// Layout of one system in GPU memory (atoms in internal, cell-sorted order):
//   x0, dlt, v, F     FP64 SoA [d][Npad]: the position is x0 + dlt, where x0
//                     is the position wrapped into the box at the last list
//                     build and dlt the displacement since then (so the
//                     rebuild trigger reads |dlt| directly);
//   sigma, inv_mass   FP64 [Npad] (inv_mass NULL means all masses are 1);
//   img               int32 SoA [d][Npad] periodic image counts;
//   id                int32 [Npad] caller index of each internal slot;
//   gs0               FP32 rows [Npad][RF]: position relative to the centre
//                     of the atom's subcell at the last build, sigma/2 in
//                     slot d (read by the list build);
//   gs[2]             FP32 rows, gs0 + (float)dlt: what the mixed-precision
//                     force loop gathers (ping-pong between MD steps);
//   gd[2]             FP64 rows [Npad][RD]: absolute position x0 + dlt and
//                     sigma/2, gathered by the FP64 force loop;
//   nbr, code         the full Verlet list: entry m of atom i sits at
//                     ((m / G) * Npad + i) * G + m % G for G lanes per atom
//                     (G = 1 is plain padded SoA), code packs for each axis
//                     the subcell offset o in {-1,0,1} of the neighbour as
//                     2 bits (o + 1), so x_i - x_j = gs_i - gs_j - o Lsc;
//   cell_*            counting-sort scratch of the binning.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hdmd {

constexpr int kMaxD = 10;
constexpr int kNRed = 16;          // reduction slots per block
#ifndef HDMD_STEP_NT
#define HDMD_STEP_NT 128
#endif
constexpr int kStepNT = HDMD_STEP_NT;   // threads per block of the force / update kernels
constexpr int kMaxLanes = 32;      // largest lanes-per-atom group

// reduction slots
enum Red {
    R_E = 0,      // sum_i e_i (each pair twice)
    R_W = 1,      // sum_i w_i (each pair twice)
    R_K2 = 2,     // sum m v^2
    R_DMAX2 = 3,  // max |dlt|^2 (max)
    R_P = 4,      // sum F.v
    R_VV = 5,     // sum v.v
    R_VF = 6,     // sum v.F/m
    R_FF = 7,     // sum (F/m).(F/m)
    R_FN = 8,     // sum F.F
    R_FMAX2 = 9,  // max |F_i|^2 (max)
    R_BAD = 10,   // non-finite seen (max)
};
__host__ __device__ constexpr bool red_is_max(int r) { return r == R_DMAX2 || r == R_FMAX2 || r == R_BAD; }

// FIRE scalar state (doubles in Flags::fire)
enum FireSlot {
    FS_DT = 0, FS_ALPHA, FS_NPOS, FS_NNEG, FS_ITER, FS_BRANCH, FS_VNORM, FS_FNORM,
    FS_STATUS, FS_FMAX, FS_E, FS_PHASE_ITER,
    FS_EPREV, FS_NFLAT, FS_FITER,   // the fractional-drop criterion
    // parameters
    FP_DTMAX, FP_DTMIN, FP_FINC, FP_FDEC, FP_ALPHA0, FP_FALPHA, FP_FTOL, FP_SWITCH,
    FP_NDELAY, FP_NNEGMAX, FP_MAXITER, FP_INITDELAY,
    FP_ETHRES, FP_FTHRES, FP_DXMAX, FP_NATOMS,
    FS_COUNT
};
enum FireStatus { FIRE_RUNNING = 0, FIRE_CONVERGED = 1, FIRE_MAXITER = 2, FIRE_NEGFAIL = 3,
                  FIRE_SWITCH = 4 };

enum ErrBits { ERR_OVERFLOW = 1, ERR_LOST = 2, ERR_BADARG = 4 };

struct Flags {
    unsigned int counter;    // last-block-done ticket
    int rebuild;             // 1: the displacement trigger fired
    int error;               // ErrBits
    int max_count;           // longest list seen by the last build
    int nbuilds;             // builds since creation
    int pad0;                // host scratch for small reads
    unsigned int disp_bits;  // max |dlt|^2 of the running step (float bits)
    int pad1;
    long long total_entries; // sum of list lengths at the last build
    long long md_step;       // MD steps since the rebuild rule was set
    double nvt_lambda;       // Berendsen factor for the next second kick
    double nvt_T;            // kinetic temperature it was computed from
    double fire[FS_COUNT];
};

struct Dev {
    int d, N, Npad, G, cap;
    int lgG;        // log2(G)
    double L, halfL, invL, skin, eps;
    int law;        // 0 harmonic, 1 Morse (Eq. (1)), 2 Mie (truncated, shifted)
    int eps_scale;  // 1: eps_ij = eps (sigma_i sigma_j)^(d/2)
    double morse_a; // Morse stiffness
    int mie_n;      // Mie exponent (law 2)
    int n;          // subcells per axis
    int ncells;
    double Lsc, invLsc;
    float Lsc_f, L_f, halfL_f;
    double *x0, *dlt, *v, *F, *sigma, *inv_mass;
    int32_t *img, *id;
    float *gs0, *gs[2];
    double *gd[2];
    // binning scratch (old order copies during a build)
    int32_t *cell_count, *cell_fill, *cell_start, *cell_of, *perm;
    int32_t *cellid;        // subcell of each internal slot at the last build
    int32_t *batch_start;   // [ncells+1] exclusive scan of ceil(count / home_batch(d))
    float hmax_f;           // largest radius (sigma_max / 2)
    double rglobal;         // > 0: one list radius sigma_max + s for every pair
    float rglobal_f;        // the same in FP32: the list build tests it per
                            // candidate chunk, where an FP64 compare would
                            // queue on the narrow FP64 pipe
    double *tx, *tv, *tsig, *tim;
    int32_t *timg, *tid;
    // lists
    int32_t *nnbr, *nbr;
    uint32_t *code;
    // reductions
    double *partials, *red;  // partials: [kNRed][maxblocks]
    int maxblocks;
    Flags *flags;
};

// home atoms held in registers by one warp of the list build
// (4 for every d: measured against 2, 3, 6 and 8, it leaves registers for
// six resident blocks per SM, which hides the latency of the row loads)
#ifndef HDMD_HOME_BATCH_LO
#define HDMD_HOME_BATCH_LO 4
#endif
__host__ __device__ constexpr int home_batch(int d) { return d <= 7 ? HDMD_HOME_BATCH_LO : 4; }

template <int D> struct Rows {
    static constexpr int RF = (D + 1 + 3) & ~3;   // floats per FP32 row
    static constexpr int RD = (D + 1 + 1) & ~1;   // doubles per FP64 row
};

__host__ __device__ inline int pow_int(int b, int e) { int r = 1; for (int k = 0; k < e; ++k) r *= b; return r; }

// entry m of atom i (G = 1 << lgG lanes per atom)
__device__ __forceinline__ int64_t list_pos(int m, int i, int Npad, int lgG) {
    return (((int64_t)(m >> lgG) * Npad + i) << lgG) + (m & ((1 << lgG) - 1));
}

// Deterministic grid reduction.  Each block reduces its threads' nslots
// partial values (sums, or maxima for the red_is_max slots) and stores them
// at dv.partials[slot * maxblocks + block]; the last block to finish (ticket
// counter, no waiting) folds all blocks' values in a fixed order into
// dv.red[slot].  Returns true in every thread of the last block.
template <int NT>
__device__ bool block_reduce_and_fold(const Dev &dv, double (&acc)[kNRed], int nslots,
                                      int maxblocks, double *sh /* [NT/32][kNRed] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r < nslots; ++r) {
        double a = acc[r];
        for (int o = 16; o > 0; o >>= 1) {
            double b = __shfl_xor_sync(0xffffffffu, a, o);
            a = red_is_max(r) ? fmax(a, b) : a + b;
        }
        if (lane == 0) sh[warp * kNRed + r] = a;
    }
    __syncthreads();
    if (threadIdx.x < nslots) {
        const int r = threadIdx.x;
        double a = sh[r];
        for (int w = 1; w < NT / 32; ++w) a = red_is_max(r) ? fmax(a, sh[w * kNRed + r]) : a + sh[w * kNRed + r];
        dv.partials[(size_t)r * maxblocks + blockIdx.x] = a;
    }
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(&dv.flags->counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int r = 0; r < nslots; ++r) {
        double a = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += NT) {
            double x = __ldcg(dv.partials + (size_t)r * maxblocks + b);
            a = red_is_max(r) ? fmax(a, x) : a + x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            double b = __shfl_xor_sync(0xffffffffu, a, o);
            a = red_is_max(r) ? fmax(a, b) : a + b;
        }
        if (lane == 0) sh[warp * kNRed + r] = a;
    }
    __syncthreads();
    if (threadIdx.x < nslots) {
        const int r = threadIdx.x;
        double a = sh[r];
        for (int w = 1; w < NT / 32; ++w) a = red_is_max(r) ? fmax(a, sh[w * kNRed + r]) : a + sh[w * kNRed + r];
        dv.red[r] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) dv.flags->counter = 0u;
    return true;
}

}  // namespace hdmd
