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
//                     2 bits (o + 1), so x_i - x_j = gs_i - gs_j - o Lsc.
//                     Packed form (pack_sh > 0, when the bits fit): one
//                     32-bit word per entry, the neighbour's index in the
//                     low pack_sh bits and above them its stencil position
//                     s = sum_k (o_k + 1) 3^k; code is then unused;
//   cell_*            counting-sort scratch of the binning.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

// Streaming (evict-first) loads and stores for the per-atom data a step reads
// and writes once; HDMD_STREAM_HINTS=0 builds them as plain accesses.
#ifndef HDMD_STREAM_HINTS
#define HDMD_STREAM_HINTS 0
#endif
#if HDMD_STREAM_HINTS
#define HDMD_LDS(p) __ldcs(p)
#define HDMD_STS(p, v) __stcs((p), (v))
#else
#define HDMD_LDS(p) (*(p))
#define HDMD_STS(p, v) (*(p) = (v))
#endif
// Packed one-word list entries where the bits fit; HDMD_PACK_LISTS=0 keeps
// the index and code arrays for every system.
#ifndef HDMD_PACK_LISTS
#define HDMD_PACK_LISTS 1
#endif

namespace hdmd {

constexpr int kMaxD = 10;
constexpr int kNRed = 16;          // reduction slots per block
#ifndef HDMD_STEP_NT
#define HDMD_STEP_NT 128
#endif
constexpr int kStepNT = HDMD_STEP_NT;   // threads per block of the force / update kernels
constexpr int kMaxLanes = 32;      // largest lanes-per-atom group
constexpr int kResNT = 1024;       // threads per block of the resident MD kernel
constexpr int kResMaxGrid = 1024;  // most blocks of the resident MD kernel
// step words of the resident MD kernel, one per 128-byte line: every block
// polls every word each step, and words that share a line queue on it
constexpr int kResWordStride = 16;

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

enum ErrBits { ERR_OVERFLOW = 1, ERR_LOST = 2, ERR_BADARG = 4, ERR_TIMEOUT = 8 };

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
    long long res_left;      // MD steps left for the resident kernel in this call
    unsigned int res_tick;   // steps the resident kernel has ever run (step words)
    int pad2;
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
    uint32_t idx_mask;   // index bits of an entry (every bit without packing)
    int pack_sh;         // > 0: packed entries, stencil position above bit pack_sh
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

// bits of a stencil position s < 3^d, ceil(log2(3^d))
__host__ __device__ constexpr int stencil_bits(int d) {
    return d <= 0 ? 0 : (d == 1 ? 2 : (d == 2 ? 4 : (d == 3 ? 5 : (d == 4 ? 7 : (d == 5 ? 8 :
           (d == 6 ? 10 : (d == 7 ? 12 : (d == 8 ? 13 : (d == 9 ? 15 : 16)))))))));
}

// stencil position of a 2-bit-per-axis offset code: s = sum_k c_k 3^k,
// c_k = o_k + 1 the 2-bit field of axis k
template <int D>
__device__ __forceinline__ uint32_t code_to_stencil(uint32_t code) {
    uint32_t s = 0;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) s = s * 3u + ((code >> (2 * k)) & 3u);
    return s;
}

// the 2-bit-per-axis offset code of a stencil position (inverse of
// code_to_stencil)
template <int D>
__device__ __forceinline__ uint32_t stencil_to_code(uint32_t s) {
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        c |= (s % 3u) << (2 * k);
        s /= 3u;
    }
    return c;
}

__host__ __device__ constexpr int pow3(int d) { return d <= 0 ? 1 : 3 * pow3(d - 1); }

// Conversions between IEEE-754 binary32 and binary64 written on the bit
// fields (sign, biased exponent, significand), so that they run on the
// integer pipe instead of the narrow FP64 pipe of this GPU.  Both follow the
// standard's definitions: binary32 -> binary64 is exact; binary64 -> binary32
// rounds to nearest, ties to even, with overflow to infinity and gradual
// underflow to subnormals; NaN stays NaN.  Host-callable too, so that a CPU
// test can hold them against the host's own conversions.
__host__ __device__ __forceinline__ uint32_t bits_f32(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float f32_bits(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
__host__ __device__ __forceinline__ uint64_t bits_f64(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
#endif
}
__host__ __device__ __forceinline__ double f64_bits(uint64_t u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, 8);
    return x;
#endif
}
__host__ __device__ __forceinline__ int lead_zeros32(uint32_t m) {
#ifdef __CUDA_ARCH__
    return __clz(m);
#else
    int k = 0;
    while (k < 32 && !(m & (0x80000000u >> k))) ++k;
    return k;
#endif
}

__host__ __device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t u = bits_f32(f);
    const uint32_t sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    uint32_t hi, lo;
    if (e != 0u && e != 0xffu) {               // normal: rebias 127 -> 1023
        hi = sign | ((e + 896u) << 20) | (m >> 3);
        lo = m << 29;
    } else if (e == 0xffu) {                   // infinity, NaN
        hi = sign | 0x7ff00000u | (m >> 3);
        lo = m << 29;
    } else if (m == 0u) {                      // signed zero
        hi = sign;
        lo = 0u;
    } else {                                   // subnormal: normalise
        const int k = lead_zeros32(m) - 8;     // shifts that bring bit 23 up
        const uint32_t mn = (m << k) & 0x7fffffu;
        hi = sign | ((uint32_t)(897 - k) << 20) | (mn >> 3);
        lo = mn << 29;
    }
    return f64_bits(((uint64_t)hi << 32) | lo);
}

__host__ __device__ __forceinline__ float f64_to_f32(double x) {
    const uint64_t bx = bits_f64(x);
    const uint32_t hi = (uint32_t)(bx >> 32), lo = (uint32_t)bx;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    const uint32_t m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);   // the kept 23 bits
    const uint32_t rest = lo & 0x1fffffffu;                      // the 29 dropped bits
    if (e == 0x7ff)                                              // infinity, NaN
        return f32_bits(sign | 0x7f800000u | m23 | ((m23 | rest) ? 0x400000u : 0u));
    const int ef = e - 896;
    if (ef >= 1) {
        if (ef >= 255) return f32_bits(sign | 0x7f800000u);
        uint32_t r = sign | ((uint32_t)ef << 23) | m23;
        r += (rest > 0x10000000u || (rest == 0x10000000u && (m23 & 1u))) ? 1u : 0u;
        return f32_bits(r);   // a carry into the exponent is the rounded value
    }
    // binary32 subnormal or zero: significand with its leading 1, shifted
    if (e == 0) return f32_bits(sign);   // binary64 zero or subnormal: below 2^-1022
    const uint64_t M = ((uint64_t)(0x100000u | (hi & 0xfffffu)) << 32) | lo;   // 53 bits
    const int sh = 926 - e;                     // >= 30
    if (sh >= 64) return f32_bits(sign);
    const uint64_t q = M >> sh, rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    const uint32_t r = (uint32_t)q + ((rem > half || (rem == half && (q & 1ull))) ? 1u : 0u);
    return f32_bits(sign | r);
}

// One FP32 row (RF floats, RF * 4-byte aligned, allocations 256-byte aligned)
// into registers.  A row of 8 floats is one 32-byte sector: one 256-bit load
// per lane, so a warp's gather of 32 scattered rows costs the L1 one tag
// look-up per row instead of two.  NC: the rows do not change while the
// kernel runs (non-coherent read-only path); otherwise they are read from L2
// (.cg), because other blocks rewrite them during the kernel.
#ifndef HDMD_ROW_V8
#define HDMD_ROW_V8 1
#endif
template <int RF, bool NC>
__device__ __forceinline__ void load_row(const float *p, float (&r)[RF]) {
#if HDMD_ROW_V8
    if constexpr (RF == 8) {
        if constexpr (NC)
            asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]),
                  "=f"(r[7])
                : "l"(p));
        else
            asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]),
                           "=f"(r[6]), "=f"(r[7])
                         : "l"(p));
        return;
    }
#endif
    const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int q = 0; q < RF / 4; ++q) {
        const float4 t = NC ? __ldg(p4 + q) : __ldcg(p4 + q);
        r[4 * q] = t.x; r[4 * q + 1] = t.y; r[4 * q + 2] = t.z; r[4 * q + 3] = t.w;
    }
}

#ifndef HDMD_INT_CVT
#define HDMD_INT_CVT 1
#endif
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float f) {
#if HDMD_INT_CVT
    return f32_to_f64(f);
#else
    return (double)f;
#endif
}
__device__ __forceinline__ float to_f32(double x) {
#if HDMD_INT_CVT
    return f64_to_f32(x);
#else
    return (float)x;
#endif
}

// Largest d whose packed entries are decoded through a shared-memory table
// of 3^d codes (2.9 KB at d = 6); larger d keep the two arrays.
constexpr int kMaxPackD = 6;

// o_k = c_k - 1 of axis k as a float, c_k the 2-bit field of the code:
// 2^23 + 2^22 + c_k has c_k in its last significand bits, and subtracting
// 2^23 + 2^22 + 1 leaves c_k - 1 exactly (no integer-to-float conversion)
__device__ __forceinline__ float code_offset(uint32_t code, int k) {
    return __uint_as_float(0x4B400000u | ((code >> (2 * k)) & 3u)) - 12582913.0f;
}

// the list entry written for neighbour j with offset code `code`
template <int D>
__device__ __forceinline__ uint32_t pack_entry(const Dev &dv, int j, uint32_t code) {
    return (uint32_t)j | (code_to_stencil<D>(code) << dv.pack_sh);
}

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
