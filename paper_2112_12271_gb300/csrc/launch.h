// launch.h -- host-side launchers of the hdmd kernels (one translation unit
// per kernel family; each dispatches the run-time d to a compile-time D).
#pragma once
#include "common.cuh"

namespace hdmd {

#define HDMD_DISPATCH_D(d, FN, ...)                    \
    switch (d) {                                       \
        case 2: FN<2>(__VA_ARGS__); break;             \
        case 3: FN<3>(__VA_ARGS__); break;             \
        case 4: FN<4>(__VA_ARGS__); break;             \
        case 5: FN<5>(__VA_ARGS__); break;             \
        case 6: FN<6>(__VA_ARGS__); break;             \
        case 7: FN<7>(__VA_ARGS__); break;             \
        case 8: FN<8>(__VA_ARGS__); break;             \
        case 9: FN<9>(__VA_ARGS__); break;             \
        case 10: FN<10>(__VA_ARGS__); break;           \
        default: break;                                \
    }

constexpr int kRowFloats(int d) { return (d + 1 + 3) & ~3; }
constexpr int kRowDoubles(int d) { return (d + 1 + 1) & ~1; }

// ---- kernels_bin.cu
// caller-order row-major staging buffers -> internal SoA (identity order)
void launch_import(const Dev &dv, const double *x_rm, const double *v_rm, const double *mass,
                   cudaStream_t s);
void launch_import_sigma(const Dev &dv, const double *sig, cudaStream_t s);
// internal -> caller-order row-major (wrapped x, img, v, F, sigma); nullable outputs
void launch_export(const Dev &dv, double *x_rm, int32_t *img_rm, double *v_rm, double *f_rm,
                   double *sig, cudaStream_t s);
// observables (kernels_obs.cu): reference = current unwrapped positions in
// caller order; displacement sums into dv.red[0..2], Z count into
// dv.red[R_P], G_s counts into hist
void launch_reference(const Dev &dv, double *ref, cudaStream_t s);
// Berendsen barostat: x <- mu x for every atom (kernels_obs.cu)
void launch_scale_positions(const Dev &dv, double mu, cudaStream_t s);
void launch_observe(const Dev &dv, const double *ref, double a2, int nbins, double inv_w,
                    unsigned int *hist, int want_z, cudaStream_t s);
// the whole list build: wrap + bin + counting sort + reorder + Verlet lists.
// buf: which gather buffer (0/1) receives the fresh rows; guarded: kernels
// return at once unless flags->rebuild is set.
void launch_rebuild(const Dev &dv, int buf, bool guarded, cudaStream_t s);
// displacement trigger without moving atoms: sets flags->rebuild
void launch_check_trigger(const Dev &dv, cudaStream_t s);
// list entries (internal order, G layout) -> caller order, for get_neighbors
void launch_list_export(const Dev &dv, int32_t *counts_out, int32_t *idx_out,
                        const int64_t *offsets, cudaStream_t s);

// ---- kernels_force.cu
struct StepCfg {
    int compute_force;   // 1: F from the list; 0: F read from dv.F
    int fp64_pairs;      // 1: FP64 pair arithmetic (gathers gd), 0: FP32 (gathers gs)
    int in_buf, out_buf; // gather rows read / written
    int kick2;           // v += dt/2 F/m (end of a step)
    int kick1_drift;     // v += dt/2 F/m; x += dt v (start of the next step)
    int store_F;         // keep F in dv.F
    int thermo;          // reduce E, W, K
    int fire_red;        // reduce P, v.v, v.F/m, F.F/m^2, F.F, max|F_i|^2 and run
                         // the FIRE scalar update in the last block
    double dt, halfdt;
    int rule;            // list rebuild rule: 0 exact (2 max|dx| > s), 1 the paper's
    int n_bet;           // the paper's rule is checked every n_bet steps
    int nvt;             // Berendsen NVT: second kick scaled by flags->nvt_lambda
    double nvt_rate;     // dt / tau
    double nvt_T;        // target temperature
    unsigned long long cond_rebuild;  // graph conditional set to the trigger (0: none)
    unsigned long long cond_loop;     // FIRE while-conditional (0: none)
};
void launch_step(const Dev &dv, const StepCfg &cfg, cudaStream_t s);
// gather rows of buffer buf rewritten from x0 + dlt
void launch_rows(const Dev &dv, int buf, int want32, int want64, cudaStream_t s);
// FIRE per-atom update from the scalars left in flags->fire by the last
// force reduction; writes gather rows of buffer 0 (FP32 and/or FP64)
void launch_fire_update(const Dev &dv, int write_fp64_rows, unsigned long long cond_rebuild,
                        cudaStream_t s);

// ---- kernels_resident.cu
struct ResCfg {
    double dt, halfdt;
    int in_buf;            // rows of the first step (and, on return, of the last)
    int nvt;               // Berendsen NVT
    double nvt_rate, nvt_T;
    int na_cap;            // atoms per block, at most (shared-memory layout)
    int list_cap;          // list words per block held in shared memory
    long long spin_limit;  // polls of a step word before ERR_TIMEOUT
    unsigned long long *sync;   // [2][grid] step words (tick << 32 | max |dlt|^2 bits),
                                // kResWordStride words apart
    double *kin;                // [2][grid] NVT partial sums
    unsigned long long cond_loop, cond_rebuild;   // graph conditionals (0: none)
};
// shared-memory bytes of the per-atom arrays of the resident kernel
size_t resident_fixed_smem(int d, int na_cap, bool pack);
cudaError_t launch_md_resident(const Dev &dv, const ResCfg &rc, int grid, size_t smem, cudaStream_t s);
cudaError_t resident_occupancy(const Dev &dv, size_t smem, int *blocks_per_sm);
// steps the next resident launches may run (flags->res_left)
void launch_set_res_left(const Dev &dv, long long nsteps, cudaStream_t s);

// ---- kernels_swap.cu
struct SwapDev {
    int npairs;
    int32_t *ids;        // [npairs][2] caller ids of the candidates
    double *u;           // [npairs] Metropolis uniforms
    int32_t *pairs;      // [npairs][2] internal slots
    int8_t *state;       // 0 pending, 1 rejected, 2 accepted
    unsigned long long *owner;   // [Npad] (round tag << 32 | pair) claims
    int32_t *slot_of;    // [Npad] caller id -> internal slot
    int32_t *slist;      // [2 npairs][scap] atoms within the largest diameter
    int32_t *scount;     // [2 npairs]
    int scap;
    int *overflow;       // swap-list overflow: longest list seen
    unsigned long long *nacc;   // accepted exchanges
    int *npend;          // pending pairs counted by the last round
    double T, rcut;      // temperature; swap-list radius (largest diameter)
};
// candidates from Philox4x32-10 (seeded) -> ids, u
void launch_swap_draw(const SwapDev &sw, uint64_t seed, int sweep, int N, cudaStream_t s);
// ids -> internal slots, state reset, swap lists built
void launch_swap_prepare(const Dev &dv, const SwapDev &sw, int buf, cudaStream_t s);
// one priority round: claim then execute every pair with no earlier pending conflict
void launch_swap_round(const Dev &dv, const SwapDev &sw, unsigned round, cudaStream_t s);

}  // namespace hdmd
