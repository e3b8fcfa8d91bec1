// kernels_resident.cu -- velocity-Verlet MD (Sec. II.B leapfrog, kick-drift-
// kick) with each block's share of the system resident in shared memory for
// many consecutive steps, one cooperative launch per list (Sec. II.C: the
// list holds until the displacement trigger fires).
//
// The system is cut into gridDim.x contiguous ranges of atoms (cell order).
// At launch each block copies its atoms' velocities and displacements (FP64),
// their build-time and current FP32 rows and their Verlet lists into shared
// memory.  Each step then reads from global memory only the FP32 rows of the
// neighbours (through L2: ld.global.cg, since other blocks rewrite them every
// step) and writes its own atoms' new rows:
//   phase A  pair forces over the list (the FP32 pair path of dev_force.cuh,
//            same lanes per atom, entry order and lane sums as the grid
//            kernel; the atoms taken longest list first);
//   phase B  the merged kicks (v += dt F/m, or the Berendsen form) and the
//            drift dlt += dt v in FP64 over (atom, axis) items, new rows
//            gs0 + (float) dlt out;
//   phase C  per-atom |dlt|^2 summed in axis order, the block's
//            maximum (and its NVT partial sum m v^2) published in a step word.
// Blocks wait for every block's word of the step (bounded spins: a wait that
// runs out sets ERR_TIMEOUT and the kernel returns), so every block sees the
// same maximum and takes the same decision: continue, or stop because the
// trigger 2 max|dlt| > s fired (or the step budget is spent).  On exit the
// state goes back to global memory and, inside a CUDA graph, the loop and
// rebuild conditionals are set.  The arithmetic of a step is that of k_step,
// so an NVE trajectory has the same bits as the one-launch-per-step path.
#include <mutex>
#include <type_traits>

#include "dev_force.cuh"
#include "launch.h"

namespace hdmd {
namespace {

constexpr int RT = kResNT;

#ifndef HDMD_RES_UNROLL
#define HDMD_RES_UNROLL 2   // list entries in flight per lane (2, 3, 4 measured)
#endif

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// pair forces of local atom a: entries from shared memory (SMEM) or from the
// global list, neighbour rows from L2
template <int D, typename FT, int LAW, bool PACK, bool SMEM>
__device__ __forceinline__ void res_forces(const Dev &dv, const float *__restrict__ gin, int a,
                                           int i, int g, int lgG, const float *sRow,
                                           const int *sOff, const uint32_t *sList,
                                           const uint32_t *sCode, const uint32_t *sTab,
                                           FT (&f)[D], FT &e, FT &w) {
    constexpr int RF = Rows<D>::RF;
    constexpr int U = HDMD_RES_UNROLL;
    const int G = 1 << lgG;
    const int nn = sOff[a + 1] - sOff[a];
    float xi[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xi[k] = sRow[a * RF + k];
    const float hi = sRow[a * RF + D];
    const float Lsc = dv.Lsc_f, eps = (float)dv.eps, ma = (float)dv.morse_a;
    const int scale = dv.eps_scale;
    const uint32_t *nbg = reinterpret_cast<const uint32_t *>(dv.nbr);
    for (int m0 = g; m0 < nn; m0 += U * G) {
        int jv[U];
        uint32_t cv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int m = m0 + u * G;
            uint32_t ent = 0u, code = 0u;
            if (m < nn) {
                if (SMEM) {
                    ent = sList[sOff[a] + m];
                    if (!PACK) code = sCode[sOff[a] + m];
                } else {
                    const int64_t pos = list_pos(m, i, dv.Npad, lgG);
                    ent = nbg[pos];
                    if (!PACK) code = dv.code[pos];
                }
            }
            jv[u] = m < nn ? (int)(PACK ? (ent & dv.idx_mask) : ent) : -1;
            cv[u] = PACK ? sTab[m < nn ? ent >> dv.pack_sh : 0u] : code;
        }
        float rj[U][RF];
#pragma unroll
        for (int u = 0; u < U; ++u) load_row<RF, false>(gin + (size_t)(jv[u] >= 0 ? jv[u] : i) * RF, rj[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jv[u] < 0) continue;
            // the scalar form of entry_dx (the same bits; measured faster here)
            float dx[D], r2 = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float t = fmaf(-code_offset(cv[u], k), Lsc, xi[k] - rj[u][k]);
                dx[k] = t;
                r2 = fmaf(t, t, r2);
            }
            pair_term_f32<D, FT, LAW>(dv, dx, r2, hi, rj[u][D], eps, ma, scale, f, e, w);
        }
    }
}

template <int D, int LAW, bool PACK>
__global__ void __launch_bounds__(RT, 1) k_md_resident(Dev dv, ResCfg rc) {
    constexpr int RF = Rows<D>::RF;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_wmax[RT / 32];   // the block's own maximum, by warp
    __shared__ unsigned s_gmax[RT / 32];   // maxima read from the step words, by warp
                                           // (separate: thread 0 may still read s_wmax)
    __shared__ double s_kinv[RT];   // the blocks' NVT partials of the step, by block
    __shared__ double s_wsum[RT / 32];
    __shared__ double s_lam;
    __shared__ int s_trig, s_lost;
    __shared__ int s_stop, s_tout, s_smem;

    const int nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int i0 = (int)((long long)dv.N * b / nb), i1 = (int)((long long)dv.N * (b + 1) / nb);
    const int na = i1 - i0, nc = rc.na_cap;
    const int G = dv.G, lgG = dv.lgG, Np = dv.Npad;

    double *sV = reinterpret_cast<double *>(smem);            // [nc][D]
    double *sDl = sV + (size_t)D * nc;                        // [nc][D]
    double *sIm = sDl + (size_t)D * nc;                       // [nc]
    float *sRow = reinterpret_cast<float *>(sIm + nc + (nc & 1));   // [nc][RF] current rows (16-B aligned)
    float *sG0 = sRow + (size_t)nc * RF;                      // [nc][RF] build-time rows
    float *sF = sG0 + (size_t)nc * RF;                        // [nc][D] forces, then (float) dlt
    int *sOff = reinterpret_cast<int *>(sF + (size_t)nc * D); // [nc + 1] list offsets
    int *sOrd = sOff + nc + 1;                                // [nc] atoms by list length
    uint32_t *sTab = reinterpret_cast<uint32_t *>(sOrd + nc);       // [3^D] codes (PACK)
    uint32_t *sList = sTab + (PACK ? pow3(D) : 0);                   // [list_cap]
    uint32_t *sCode = sList + rc.list_cap;                           // [list_cap] (!PACK)

    const long long left0 = dv.flags->res_left;
    const unsigned tick0 = dv.flags->res_tick;
    const int err0 = dv.flags->error;
    if (left0 <= 0 || (err0 & (ERR_OVERFLOW | ERR_LOST | ERR_TIMEOUT))) {
        if (b == 0 && tid == 0) {
            dv.flags->rebuild = 0;
            if (rc.cond_loop) cudaGraphSetConditional(rc.cond_loop, 0u);
            if (rc.cond_rebuild) cudaGraphSetConditional(rc.cond_rebuild, 0u);
        }
        return;
    }

    // ---- load the block's atoms
    for (int t = tid; t < na * D; t += RT) {
        const int k = t / na, a = t - k * na;
        const size_t o = (size_t)k * Np + i0 + a;
        sV[a * D + k] = dv.v[o];
        sDl[a * D + k] = dv.dlt[o];
    }
    if (dv.inv_mass)
        for (int a = tid; a < na; a += RT) sIm[a] = dv.inv_mass[i0 + a];
    {
        const float *gr = dv.gs[rc.in_buf] + (size_t)i0 * RF, *g0 = dv.gs0 + (size_t)i0 * RF;
        for (int t = tid; t < na * RF; t += RT) {
            sRow[t] = gr[t];
            sG0[t] = g0[t];
        }
    }
    if (RF > D) {
        // the radius (and padding) of the rows in the other buffer: steps
        // rewrite only the coordinates
        float *go = dv.gs[rc.in_buf ^ 1] + (size_t)i0 * RF;
        const float *g0 = dv.gs0 + (size_t)i0 * RF;
        for (int t = tid; t < na * (RF - D); t += RT) {
            const int a = t / (RF - D), c = D + (t - a * (RF - D));
            go[a * RF + c] = g0[a * RF + c];
        }
    }
    if (PACK)
        for (int t = tid; t < pow3(D); t += RT) sTab[t] = stencil_to_code<D>((uint32_t)t);
    // list offsets: exclusive prefix of the list lengths (warp 0, chunks of atoms)
    if (warp == 0) {
        const int per = (na + 31) / 32, lo = min(lane * per, na), hi = min(lo + per, na);
        int sum = 0;
        for (int a = lo; a < hi; ++a) sum += dv.nnbr[i0 + a];
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int run = incl - sum;
        for (int a = lo; a < hi; ++a) {
            sOff[a] = run;
            run += dv.nnbr[i0 + a];
        }
        if (lane == 31) {
            sOff[na] = incl;
            s_smem = incl <= rc.list_cap ? 1 : 0;
        }
    }
    __syncthreads();
    // lane order of phase A: the block's atoms by list length, longest first
    // (ties by index), so that the atoms of a warp have lists of about the
    // same length and few lanes idle at the end of the shortest ones; every
    // atom keeps its own lanes and entry order, so its force has the same bits
    for (int a = tid; a < na; a += RT) {
        const int la = sOff[a + 1] - sOff[a];
        int r = 0;
        for (int q = 0; q < na; ++q) {
            const int lq = sOff[q + 1] - sOff[q];
            r += (lq > la) || (lq == la && q < a);
        }
        sOrd[r] = a;
    }
    const bool in_smem = s_smem != 0;
    if (in_smem) {
        const int apr = RT >> lgG;
        for (int a0 = 0; a0 < na; a0 += apr) {
            const int a = a0 + (tid >> lgG), g = tid & (G - 1);
            if (a >= na) continue;
            const int nn = sOff[a + 1] - sOff[a];
            for (int m = g; m < nn; m += G) {
                const int64_t pos = list_pos(m, i0 + a, Np, lgG);
                sList[sOff[a] + m] = (uint32_t)dv.nbr[pos];
                if (!PACK) sCode[sOff[a] + m] = dv.code[pos];
            }
        }
    }
    if (tid == 0) s_lam = dv.flags->nvt_lambda;
    __syncthreads();

    long long left = left0;
    int steps = 0, trig = 0, lost = 0, tout = 0;
    const double dt = rc.dt, hdt = rc.halfdt;
    const bool nvt = rc.nvt != 0;
    const float s2 = (float)(dv.skin * dv.skin) * (1.0f - 1e-5f);
    while (left > 0) {
        const int pin = rc.in_buf ^ (steps & 1), pout = pin ^ 1;
        const float *gin = dv.gs[pin];
        // ---- phases A and B, warp by warp: a warp's atoms (slots of the
        // lane order) get their pair forces, and the same warp at once takes
        // their merged kicks (v += dt F/m, or the Berendsen form) and drift in
        // FP64 (the arithmetic of k_step) over (atom, axis) items, with no
        // block barrier between: the slow FP64 pipe works beside the other
        // warps' row gathers.  (float) dlt replaces the force in sF; the new
        // row coordinate goes to sRow and straight out to the other row buffer.
        // Then |dlt|^2 of each atom, summed by one lane in axis order (the
        // trigger repeats bit for bit).
        double kin = 0.0;
        unsigned mb = 0u;
        {
            const int apr = RT >> lgG, apw = 32 >> lgG;   // atom slots per pass, per warp
            const double lam = s_lam;
            const bool masses = dv.inv_mass != nullptr;
            float *go = dv.gs[pout] + (size_t)i0 * RF;
            for (int a0 = 0; a0 < na; a0 += apr) {
                const int slot = a0 + (tid >> lgG), g = tid & (G - 1);
                const bool live = slot < na;
                const int a = live ? sOrd[slot] : 0;
                float f[D];
#pragma unroll
                for (int k = 0; k < D; ++k) f[k] = 0.f;
                float e = 0.f, w = 0.f;
                if (live) {
                    if (in_smem)
                        res_forces<D, float, LAW, PACK, true>(dv, gin, a, i0 + a, g, lgG, sRow, sOff, sList,
                                                              sCode, sTab, f, e, w);
                    else
                        res_forces<D, float, LAW, PACK, false>(dv, gin, a, i0 + a, g, lgG, sRow, sOff, sList,
                                                               sCode, sTab, f, e, w);
                }
                for (int o = G >> 1; o > 0; o >>= 1) {
#pragma unroll
                    for (int k = 0; k < D; ++k) f[k] += __shfl_xor_sync(0xffffffffu, f[k], o);
                }
                if (g == 0 && live) {
#pragma unroll
                    for (int k = 0; k < D; ++k) sF[a * D + k] = f[k];
                }
                __syncwarp();
                const int s0 = a0 + warp * apw;   // this warp's first slot
                // (two copies of the loop: without masses there is no multiply
                // by 1/m at all, not even one the compiler might speculate)
                auto items = [&](auto with_mass) {
                    constexpr bool MASS = decltype(with_mass)::value;
                    for (int q = lane; q < apw * D; q += 32) {
                        const int qa = q / D, k = q - qa * D;
                        if (s0 + qa >= na) break;
                        const int aa = sOrd[s0 + qa], t = aa * D + k;
                        const double F = to_f64(sF[t]);
                        double Fm = F, im = 1.0;
                        if constexpr (MASS) {
                            im = sIm[aa];
                            Fm = F * im;
                        }
                        double v = sV[t];
                        if (nvt) {
                            const double vf = (v + hdt * Fm) * lam;
                            kin += vf * vf / im;
                            v = vf + hdt * Fm;
                        } else {
                            v += dt * Fm;
                        }
                        const double dl = sDl[t] + dt * v;
                        sDl[t] = dl;
                        sV[t] = v;
                        const float fl = to_f32(dl);
                        sF[t] = fl;
                        const float r = sG0[aa * RF + k] + fl;
                        sRow[aa * RF + k] = r;
                        go[aa * RF + k] = r;
                    }
                };
                if (masses) items(std::true_type{});
                else items(std::false_type{});
                __syncwarp();
                if (lane < apw && s0 + lane < na) {
                    const int aa = sOrd[s0 + lane];
                    float d2 = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k) d2 = fmaf(sF[aa * D + k], sF[aa * D + k], d2);
                    mb = max(mb, __float_as_uint(d2));
                }
            }
        }
        mb = __reduce_max_sync(0xffffffffu, mb);
        double ks = kin;
        if (nvt)
            for (int o = 16; o > 0; o >>= 1) ks += __shfl_xor_sync(0xffffffffu, ks, o);
        if (lane == 0) {
            s_wmax[warp] = mb;
            s_wsum[warp] = ks;
        }
        // ---- step word
        __syncthreads();
        const unsigned tick = tick0 + (unsigned)steps + 1u;
        const int par = (int)(tick & 1u);
        if (tid == 0) {
            unsigned m = 0u;
            for (int q = 0; q < RT / 32; ++q) m = max(m, s_wmax[q]);
            if (nvt) {
                // a chain of dependent FP64 adds (slow on this pipe): NVT only
                double kb = 0.0;
                for (int q = 0; q < RT / 32; ++q) kb += s_wsum[q];
                rc.kin[(size_t)par * nb + b] = kb;
            }
            // a release at GPU scope: the block's row stores, ordered before
            // this thread by the barrier above, become visible before the word
            // (no separate fence: the release is cumulative over them)
            st_release_u64(rc.sync + ((size_t)par * nb + b) * kResWordStride, ((unsigned long long)tick << 32) | m);
        }
        // ---- wait for every block's word of this step
        unsigned gm = 0u;
        int to = 0;
        for (int c = tid; c < nb; c += RT) {
            unsigned long long wv = 0ull;
            long long it = 0;
            for (;;) {
                wv = ld_acquire_u64(rc.sync + ((size_t)par * nb + c) * kResWordStride);
                if ((unsigned)(wv >> 32) == tick) break;
                if (++it > rc.spin_limit) { to = 1; break; }
                if (it > 64) __nanosleep(32);
            }
            gm = max(gm, (unsigned)wv);
            // written before the word's release, so visible after its acquire
            if (nvt) s_kinv[c] = __ldcg(rc.kin + (size_t)par * nb + c);
        }
        // later reads of other blocks' rows, by any thread of the block, come
        // after the words' acquires: the barrier below orders the two
        gm = __reduce_max_sync(0xffffffffu, gm);
        if (lane == 0) s_gmax[warp] = gm;
        to = __syncthreads_or(to);
        if (tid == 0) {
            unsigned m = 0u;
            for (int q = 0; q < RT / 32; ++q) m = max(m, s_gmax[q]);
            s_tout = to;
            // the step's decision, taken once (the FP64 compare is slow on
            // this pipe): the trigger 2 max|dlt| > s, and a lost atom
            const float d2 = __uint_as_float(m);
            const bool finite = d2 <= 3.0e38f;
            s_trig = (4.0f * d2 > s2) || !finite;
            s_lost = !finite || 16.0 * (double)d2 > dv.L * dv.L;
            if (nvt && !to) {
                double k2 = 0.0;
                for (int c = 0; c < nb; ++c) k2 += s_kinv[c];   // block order: the same sum everywhere
                const double T = k2 / ((double)dv.d * (double)(dv.N - 1));
                dv.flags->nvt_T = T;   // (every block computes the same value)
                s_lam = T > 0.0 ? sqrt(fmax(0.0, 1.0 + rc.nvt_rate * (rc.nvt_T / T - 1.0))) : 1.0;
            }
        }
        __syncthreads();
        ++steps;
        --left;
        if (s_tout) { tout = 1; break; }
        trig = s_trig;
        lost = s_lost;
        if (trig) break;
    }

    // ---- state back to global memory; the latest rows into gs[in_buf]
    for (int t = tid; t < na * D; t += RT) {
        const int k = t / na, a = t - k * na;
        const size_t o = (size_t)k * Np + i0 + a;
        dv.v[o] = sV[a * D + k];
        dv.dlt[o] = sDl[a * D + k];
    }
    if (steps & 1) {
        float *go = dv.gs[rc.in_buf] + (size_t)i0 * RF;
        for (int t = tid; t < na * RF; t += RT) go[t] = sRow[t];
    }
    if (b == 0 && tid == 0) {
        dv.flags->res_left = left;
        // after a time-out the blocks may disagree on the step count: move the
        // tick far ahead so that no old step word matches a later step
        dv.flags->res_tick = tick0 + (unsigned)steps + (tout ? (1u << 24) : 0u);
        dv.flags->rebuild = trig;
        if (nvt) dv.flags->nvt_lambda = s_lam;
        int err = 0;
        if (lost) err |= ERR_LOST;
        if (tout) err |= ERR_TIMEOUT;
        if (err) atomicOr(&dv.flags->error, err);
        if (rc.cond_loop) cudaGraphSetConditional(rc.cond_loop, (left > 0 && !err) ? 1u : 0u);
        if (rc.cond_rebuild) cudaGraphSetConditional(rc.cond_rebuild, trig ? 1u : 0u);
    }
}

// The kernel's dynamic shared-memory limit, raised once per device to all
// that the device allows beside the kernel's static arrays (and never
// lowered), under a lock: systems on several host threads launch the same
// kernel with different sizes, and a per-launch setting would race.
template <int D, int LAW, bool PACK>
cudaError_t ensure_smem_limit() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_md_resident<D, LAW, PACK>);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_md_resident<D, LAW, PACK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

template <int D, int LAW, bool PACK>
cudaError_t launch_one(const Dev &dv, const ResCfg &rc, int grid, size_t smem, cudaStream_t s) {
    auto kern = k_md_resident<D, LAW, PACK>;
    cudaError_t e = ensure_smem_limit<D, LAW, PACK>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(RT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, dv, rc);
}

template <int D, int LAW, bool PACK>
cudaError_t occupancy_one(size_t smem, int *blocks_per_sm) {
    auto kern = k_md_resident<D, LAW, PACK>;
    cudaError_t e = ensure_smem_limit<D, LAW, PACK>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, RT, smem);
}

template <int D>
cudaError_t res_dispatch(const Dev &dv, const ResCfg *rc, int grid, size_t smem, cudaStream_t s,
                         int *occ) {
    const bool pack = D <= kMaxPackD && dv.pack_sh > 0;
    if (occ) {
        if (dv.law == 1) return pack ? occupancy_one<D, 1, (D <= kMaxPackD)>(smem, occ) : occupancy_one<D, 1, false>(smem, occ);
        if (dv.law == 2) return pack ? occupancy_one<D, 2, (D <= kMaxPackD)>(smem, occ) : occupancy_one<D, 2, false>(smem, occ);
        return pack ? occupancy_one<D, 0, (D <= kMaxPackD)>(smem, occ) : occupancy_one<D, 0, false>(smem, occ);
    }
    if (dv.law == 1) return pack ? launch_one<D, 1, (D <= kMaxPackD)>(dv, *rc, grid, smem, s) : launch_one<D, 1, false>(dv, *rc, grid, smem, s);
    if (dv.law == 2) return pack ? launch_one<D, 2, (D <= kMaxPackD)>(dv, *rc, grid, smem, s) : launch_one<D, 2, false>(dv, *rc, grid, smem, s);
    return pack ? launch_one<D, 0, (D <= kMaxPackD)>(dv, *rc, grid, smem, s) : launch_one<D, 0, false>(dv, *rc, grid, smem, s);
}

template <int D>
void res_dispatch_v(const Dev &dv, const ResCfg *rc, int grid, size_t smem, cudaStream_t s, int *occ,
                    cudaError_t *out) {
    *out = res_dispatch<D>(dv, rc, grid, smem, s, occ);
}

__global__ void k_set_res_left(Flags *fl, long long n) { fl->res_left = n; }

}  // namespace

void launch_set_res_left(const Dev &dv, long long nsteps, cudaStream_t s) {
    k_set_res_left<<<1, 1, 0, s>>>(dv.flags, nsteps);
}

size_t resident_fixed_smem(int d, int na_cap, bool pack) {
    const size_t RF = kRowFloats(d);
    size_t b = (size_t)(na_cap + (na_cap & 1)) * (2 * d * 8 + 8) + (size_t)na_cap * RF * 4 * 2 + (size_t)na_cap * d * 4 +
               (size_t)(na_cap + 1) * 4 + (size_t)na_cap * 4;
    if (pack) b += (size_t)pow3(d) * 4;
    return b;
}

cudaError_t launch_md_resident(const Dev &dv, const ResCfg &rc, int grid, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaErrorInvalidValue;
    HDMD_DISPATCH_D(dv.d, res_dispatch_v, dv, &rc, grid, smem, s, nullptr, &e);
    return e;
}

cudaError_t resident_occupancy(const Dev &dv, size_t smem, int *blocks_per_sm) {
    cudaError_t e = cudaErrorInvalidValue;
    HDMD_DISPATCH_D(dv.d, res_dispatch_v, dv, nullptr, 0, smem, nullptr, blocks_per_sm, &e);
    return e;
}

}  // namespace hdmd
