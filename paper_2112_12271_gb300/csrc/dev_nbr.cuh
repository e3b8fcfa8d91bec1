// dev_nbr.cuh -- device function of the Verlet-list build (see
// kernels_nbr.cu for the method); shared by the grid and batched kernels.
#pragma once
#include "common.cuh"

namespace hdmd {

// Lists of home batch w (one warp; lane = 0..31).  Called by the grid
// kernel below (one warp per batch) and by the batched-job kernel (the warps
// of one block loop over the batches of one job).  ALLH (n_cell >= 3 only):
// test a candidate against all home atoms branch-free before one vote,
// instead of one home atom after another; it pays where registers are
// plentiful enough for more resident warps (d <= 4), not above.
template <int D, bool WRAP, bool ALLH = false>
__device__ __forceinline__ void nbr_batch(const Dev &dv, int w, int lane) {
    constexpr int RF = Rows<D>::RF;
    constexpr int H = home_batch(D);
    // home subcell: largest c with batch_start[c] <= w
    int lo = 0, hi = dv.ncells - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (dv.batch_start[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const int c = lo;
    const int cs = dv.cell_start[c], ce = dv.cell_start[c + 1];
    const int h0 = cs + (w - dv.batch_start[c]) * H;
    const int nh = min(H, ce - h0);
    const int n = dv.n;
    int C[D];
    {
        int t = c;
#pragma unroll
        for (int k = D - 1; k >= 0; --k) { C[k] = t % n; t /= n; }
    }
    const float Lsc = dv.Lsc_f, hLsc = 0.5f * dv.Lsc_f, hL = dv.halfL_f;
    const float skin = (float)dv.skin;
    const bool glob = dv.rglobal_f > 0.f;   // one list radius for every pair
    const float band_abs = 1e-5f * Lsc * Lsc;

    // home atoms in registers (identical in every lane)
    float xh[H][D], rh[H];
    int cnt[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int i = h < nh ? h0 + h : h0;
        const float *ri = dv.gs0 + (size_t)i * RF;
#pragma unroll
        for (int k = 0; k < D; ++k) xh[h][k] = ri[k];
        rh[h] = (glob ? dv.hmax_f : ri[D]) + skin;
        cnt[h] = 0;
    }
    const float reach_pad = dv.hmax_f;   // largest candidate radius
    // n_cell >= 3: the test below is written as
    //   |r_j - x_h|^2 - (rho_j + rho_h)^2
    //     = (|r_j|^2 - rho_j^2) + (|x_h|^2 - rho_h^2) - 2 (r_j . x_h + rho_j rho_h),
    // the first bracket once per candidate, the second once per home atom, so
    // a pair test is d + 3 operations.  Its rounding error is below
    // (d + 3) u S with S = sum_k (|r_jk| + |x_hk|)^2 + (rho_j + rho_h)^2
    // <= (4d + 1) L_sc^2 (|x_hk| <= L_sc/2, |r_jk| <= 3 L_sc/2, rho_j + rho_h
    // <= L_sc); twice that widens the guard band, which stays far below
    // L_sc^2, so the FP64 recheck remains rare.
    float Bh[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        float b = -rh[h] * rh[h];
#pragma unroll
        for (int k = 0; k < D; ++k) b = fmaf(xh[h][k], xh[h][k], b);
        Bh[h] = b;
    }
    const float rcmax = 2.f * dv.hmax_f + skin;   // largest cutoff
    const float band_x = fmaf(1e-5f, rcmax * rcmax, band_abs)
                       + (float)((D + 3) * (4 * D + 1)) * 1.2e-7f * Lsc * Lsc;
    const int base = WRAP ? 3 : (n == 1 ? 1 : 2);   // distinct offsets per axis
    const int Srow = pow_int(base, D - 1);
    const int cl = C[D - 1];
    const int cl_m = cl == 0 ? n - 1 : cl - 1, cl_p = cl == n - 1 ? 0 : cl + 1;
    const unsigned allh = (1u << nh) - 1u;

    // rows of the stencil, 32 at a time: lane l works out row sr0 + l (its
    // subcell index, offset code, which home atoms can reach it and where its
    // atoms lie), then the warp walks the reachable rows one by one
    for (int sr0 = 0; sr0 < Srow; sr0 += 32) {
        const int sr = sr0 + lane;
        int Jrow = 0;
        uint32_t rcode = 0;
        unsigned amask = 0;
        int ps1 = 0, pl1 = 0, ps2 = 0, pl2 = 0, ps3 = 0, pl3 = 0;   // the row's pieces
        if (sr < Srow) {
            int off[D];
            int rem = sr;
#pragma unroll
            for (int k = D - 2; k >= 0; --k) { off[k] = rem % base - (WRAP ? 1 : 0); rem /= base; }
#pragma unroll
            for (int k = 0; k < D - 1; ++k) {
                int cj = C[k] + off[k];
                cj = cj < 0 ? cj + n : (cj >= n ? cj - n : cj);
                Jrow = Jrow * n + cj;
                rcode |= (uint32_t)(off[k] + 1) << (2 * k);
            }
            Jrow *= n;
            unsigned mlo = 0, mhi = 0;   // home atoms reaching the row's lower / upper piece
            if (WRAP) {
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    float b2 = 0.f;
#pragma unroll
                    for (int k = 0; k < D - 1; ++k) {
                        float dk = off[k] > 0 ? hLsc - xh[h][k] : (off[k] < 0 ? xh[h][k] + hLsc : 0.f);
                        dk = fmaxf(dk, 0.f);
                        b2 = fmaf(dk, dk, b2);
                    }
                    const float reach = (rh[h] + reach_pad) * (1.0f + 1e-5f) + 1e-5f;
                    const float r2 = reach * reach;
                    const float dlo = fmaxf(xh[h][D - 1] + hLsc, 0.f), dhi = fmaxf(hLsc - xh[h][D - 1], 0.f);
                    if (b2 < r2) amask |= 1u << h;
                    if (fmaf(dlo, dlo, b2) < r2) mlo |= 1u << h;
                    if (fmaf(dhi, dhi, b2) < r2) mhi |= 1u << h;
                }
                amask &= allh;
                mlo &= allh;
                mhi &= allh;
            } else {
                amask = allh;
            }
            // the row's subcells along the last axis as up to three pieces,
            // looked up here for all 32 rows at once (one round trip) rather
            // than row after row in the walk below
            if (amask) {
                if (WRAP) {   // a piece no home atom reaches along the last axis either is skipped
                    ps1 = dv.cell_start[Jrow + cl_m]; pl1 = mlo ? dv.cell_start[Jrow + cl_m + 1] - ps1 : 0;
                    ps2 = dv.cell_start[Jrow + cl];   pl2 = dv.cell_start[Jrow + cl + 1] - ps2;
                    ps3 = dv.cell_start[Jrow + cl_p]; pl3 = mhi ? dv.cell_start[Jrow + cl_p + 1] - ps3 : 0;
                } else if (n == 2) {
                    ps1 = dv.cell_start[Jrow + cl];     pl1 = dv.cell_start[Jrow + cl + 1] - ps1;
                    ps2 = dv.cell_start[Jrow + 1 - cl]; pl2 = dv.cell_start[Jrow + 2 - cl] - ps2;
                } else {   // one subcell: every atom
                    ps1 = dv.cell_start[0]; pl1 = dv.cell_start[1] - ps1;
                    ps2 = ps1;
                }
            }
        }
        unsigned rows = __ballot_sync(0xffffffffu, amask != 0);
        while (rows) {
            const int src = __ffs(rows) - 1;
            rows &= rows - 1;
            const uint32_t rc0 = __shfl_sync(0xffffffffu, rcode, src);
            const unsigned active = __shfl_sync(0xffffffffu, amask, src);
            float offL[D];   // offsets of axes 0..D-2 times L_sc (WRAP)
#pragma unroll
            for (int k = 0; k < D - 1; ++k) offL[k] = (float)((int)((rc0 >> (2 * k)) & 3u) - 1) * Lsc;
            // the row's subcells along the last axis, as up to three pieces
            const int s1 = __shfl_sync(0xffffffffu, ps1, src), l1 = __shfl_sync(0xffffffffu, pl1, src);
            const int s2 = __shfl_sync(0xffffffffu, ps2, src), l2 = __shfl_sync(0xffffffffu, pl2, src);
            const int s3 = __shfl_sync(0xffffffffu, ps3, src), l3 = __shfl_sync(0xffffffffu, pl3, src);
            const int o1 = WRAP ? -1 : 0, o2 = WRAP ? 0 : (n == 2 ? 1 : 0), o3 = 1;
            const int tot = l1 + l2 + l3;
            for (int t0 = 0; t0 < tot; t0 += 32) {
                const int t = t0 + lane;
                const bool okj = t < tot;
                int j, olast;
                if (t < l1) { j = s1 + t; olast = o1; }
                else if (t < l1 + l2) { j = s2 + (t - l1); olast = o2; }
                else { j = s3 + (t - l1 - l2); olast = o3; }
                if (!okj) { j = s1 < dv.N ? s1 : 0; olast = o1; }
                float rj[RF];
                {
                    const float4 *rj4 = reinterpret_cast<const float4 *>(dv.gs0 + (size_t)j * RF);
#pragma unroll
                    for (int q = 0; q < RF / 4; ++q) {
                        const float4 tt = __ldg(rj4 + q);
                        rj[4 * q] = tt.x; rj[4 * q + 1] = tt.y; rj[4 * q + 2] = tt.z; rj[4 * q + 3] = tt.w;
                    }
                }
                float rhoj = 0.f, Aj = 0.f;
                if (WRAP) {
#pragma unroll
                    for (int k = 0; k < D - 1; ++k) rj[k] += offL[k];
                    rj[D - 1] = fmaf((float)olast, Lsc, rj[D - 1]);
                    rhoj = glob ? dv.hmax_f : rj[D];
                    Aj = -rhoj * rhoj;
#pragma unroll
                    for (int k = 0; k < D; ++k) Aj = fmaf(rj[k], rj[k], Aj);
                }
                const uint32_t wcode = WRAP ? (rc0 | ((uint32_t)(olast + 1) << (2 * (D - 1)))) : 0u;
                if constexpr (WRAP && ALLH) {
                    // every home atom's test at once (independent chains),
                    // then one vote: most chunks hold no pair at all
                    unsigned hits = 0u, close = 0u;
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        float da = rhoj * rh[h], db = 0.f;
#pragma unroll
                        for (int k = 0; k < D; ++k) {
                            if (k & 1) db = fmaf(rj[k], xh[h][k], db);
                            else da = fmaf(rj[k], xh[h][k], da);
                        }
                        const float diff = fmaf(-2.f, da + db, Aj + Bh[h]);
                        hits |= (diff < -band_x ? 1u : 0u) << h;
                        close |= (fabsf(diff) <= band_x ? 1u : 0u) << h;
                    }
                    const unsigned self = (unsigned)(j - h0) < (unsigned)H ? 1u << (j - h0) : 0u;
                    const unsigned cand = okj ? (active & ~self) : 0u;
                    hits &= cand;
                    close &= cand;
                    while (close) {   // FP64 decision (positions are x0 at a build)
                        const int h = __ffs(close) - 1;
                        close &= close - 1;
                        const int i = h0 + h;
                        double s2d = 0.0;
                        for (int k = 0; k < D; ++k) {
                            double dx = dv.x0[(size_t)k * dv.Npad + j] - dv.x0[(size_t)k * dv.Npad + i];
                            dx -= dv.L * rint(dx * dv.invL);
                            s2d += dx * dx;
                        }
                        const double rcd = glob ? dv.rglobal
                                                : 0.5 * (dv.sigma[i] + dv.sigma[j]) + dv.skin;
                        if (s2d < rcd * rcd) hits |= 1u << h;
                    }
                    if (!__any_sync(0xffffffffu, hits != 0u)) continue;
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        if (!(active & (1u << h))) continue;   // warp-uniform
                        const bool hit = (hits >> h) & 1u;
                        const unsigned m = __ballot_sync(0xffffffffu, hit);
                        if (!m) continue;
                        if (hit) {
                            const int idx = cnt[h] + __popc(m & ((1u << lane) - 1u));
                            if (idx < dv.cap) {
                                const int64_t pos = list_pos(idx, h0 + h, dv.Npad, dv.lgG);
                                if (dv.pack_sh) {
                                    dv.nbr[pos] = (int32_t)pack_entry<D>(dv, j, wcode);
                                } else {
                                    dv.nbr[pos] = j;
                                    dv.code[pos] = wcode;
                                }
                            }
                        }
                        cnt[h] += __popc(m);
                    }
                } else {
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        if (!(active & (1u << h))) continue;   // warp-uniform
                        const int i = h0 + h;
                        bool hit = false;
                        uint32_t code = wcode;
                        if (okj && j != i) {
                            float diff, band;
                            if (WRAP) {
                                float dot = rhoj * rh[h];
#pragma unroll
                                for (int k = 0; k < D; ++k) dot = fmaf(rj[k], xh[h][k], dot);
                                diff = fmaf(-2.f, dot, Aj + Bh[h]);
                                band = band_x;
                            } else {
                                float r2 = 0.f;
                                code = 0u;
#pragma unroll
                                for (int k = 0; k < D; ++k) {
                                    const int ok = k < D - 1 ? (int)((rc0 >> (2 * k)) & 3u) - 1 : olast;   // 0 or +1
                                    float dx = rj[k] - xh[h][k];
                                    int o = ok;
                                    if (ok) {
                                        const float dp = (rj[k] + Lsc) - xh[h][k];
                                        if (dp > hL) { dx = (rj[k] - Lsc) - xh[h][k]; o = -1; }
                                        else dx = dp;
                                    } else if (n == 1) {   // L_sc = L: nearest image either way
                                        if (dx > hL) { dx = (rj[k] - Lsc) - xh[h][k]; o = -1; }
                                        else if (dx < -hL) { dx = (rj[k] + Lsc) - xh[h][k]; o = 1; }
                                    }
                                    code |= (uint32_t)(o + 1) << (2 * k);
                                    r2 = fmaf(dx, dx, r2);
                                }
                                const float rc = rh[h] + (glob ? dv.hmax_f : rj[D]);
                                const float rc2 = rc * rc;
                                diff = r2 - rc2;
                                band = band_abs + 1e-5f * rc2;
                            }
                            if (diff > band) {
                                hit = false;
                            } else if (fabsf(diff) <= band) {
                                // FP64 decision (positions are x0 at a build)
                                double s2d = 0.0;
                                for (int k = 0; k < D; ++k) {
                                    double dx = dv.x0[(size_t)k * dv.Npad + j] - dv.x0[(size_t)k * dv.Npad + i];
                                    dx -= dv.L * rint(dx * dv.invL);
                                    s2d += dx * dx;
                                }
                                const double rcd = glob ? dv.rglobal
                                                        : 0.5 * (dv.sigma[i] + dv.sigma[j]) + dv.skin;
                                hit = s2d < rcd * rcd;
                            } else {
                                hit = diff < 0.f;
                            }
                        }
                        const unsigned m = __ballot_sync(0xffffffffu, hit);
                        if (!m) continue;
                        if (hit) {
                            const int idx = cnt[h] + __popc(m & ((1u << lane) - 1u));
                            if (idx < dv.cap) {
                                const int64_t pos = list_pos(idx, i, dv.Npad, dv.lgG);
                                if (dv.pack_sh) {
                                    dv.nbr[pos] = (int32_t)pack_entry<D>(dv, j, code);
                                } else {
                                    dv.nbr[pos] = j;
                                    dv.code[pos] = code;
                                }
                            }
                        }
                        cnt[h] += __popc(m);
                    }
                }
            }
        }
    }
    if (lane < nh) {
        int cnt_l = 0;
#pragma unroll
        for (int h = 0; h < H; ++h) if (h == lane) cnt_l = cnt[h];
        const int i = h0 + lane;
        dv.nnbr[i] = min(cnt_l, dv.cap);
        if (cnt_l > dv.cap) atomicOr(&dv.flags->error, (int)ERR_OVERFLOW);
        atomicMax(&dv.flags->max_count, cnt_l);
        atomicAdd((unsigned long long *)&dv.flags->total_entries, (unsigned long long)cnt_l);
    }
}

// Lists of every atom of home subcell c (one warp; n_cell >= 3), the home
// atoms staged in shared memory (sh: 32 x home_row_floats(D) floats of this
// warp: -2 x_h, -2 rho_h and |x_h|^2 - rho_h^2, so that the test of a
// candidate is one add and D + 1 fused multiply-adds) and read by broadcast,
// the lanes carrying candidates: each candidate is tested against all home
// atoms that reach its row (the expanded test of nbr_batch, branch-free) for
// one mask of pairs inside the list radius or within the rounding band of it;
// only those pairs are looked at again (band: FP64 decision), and only a
// chunk with a hit takes the vote and the compaction.  Home atoms beyond 32
// are taken in further passes.  Entries come out in the order of nbr_batch:
// rows, then pieces, then candidates.
//
// HALF (Newton's third law): a home subcell takes the rows of the stencil
// whose first non-zero offset on axes 0..D-2 is positive, and of the row of
// zero offsets the pieces at last-axis offsets 0 and +1, the home piece only
// for the pairs i < j; each pair found is entered in both lists (offset o
// for the home atom, -o for the candidate) at slots taken by atomics on the
// counters (zeroed by the binning), and k_list_finish then sorts every list
// by neighbour index and clamps the counts: the same lists, in index order.
__host__ __device__ constexpr int home_row_floats(int D) { return (D + 2 + 3) & ~3; }

template <int D, bool HALF>
__device__ __forceinline__ void nbr_cell(const Dev &dv, int c, int lane, float *sh) {
    constexpr int RF = Rows<D>::RF, HR = home_row_floats(D);
    const int cs = dv.cell_start[c], ce = dv.cell_start[c + 1];
    const int n = dv.n;
    int C[D];
    {
        int t = c;
#pragma unroll
        for (int k = D - 1; k >= 0; --k) { C[k] = t % n; t /= n; }
    }
    const float Lsc = dv.Lsc_f, hLsc = 0.5f * dv.Lsc_f;
    const float skin = (float)dv.skin;
    const bool glob = dv.rglobal_f > 0.f;
    const float band_abs = 1e-5f * Lsc * Lsc;
    const float reach_pad = dv.hmax_f;
    const float rcmax = 2.f * dv.hmax_f + skin;
    const float band_x = fmaf(1e-5f, rcmax * rcmax, band_abs)
                       + (float)((D + 3) * (4 * D + 1)) * 1.2e-7f * Lsc * Lsc;
    const int Srow = pow_int(3, D - 1);
    const int cl = C[D - 1];
    const int cl_m = cl == 0 ? n - 1 : cl - 1, cl_p = cl == n - 1 ? 0 : cl + 1;

    for (int h0 = cs; h0 < ce; h0 += 32) {
        const int nh = min(32, ce - h0);
        const unsigned allh = nh == 32 ? 0xffffffffu : (1u << nh) - 1u;
        // stage the home atoms: coordinates, list radius, |x|^2 - rho^2
        __syncwarp();
        if (lane < nh) {
            const float *ri = dv.gs0 + (size_t)(h0 + lane) * RF;
            float *hr = sh + lane * HR;
            const float rh = (glob ? dv.hmax_f : ri[D]) + skin;
            float b = -rh * rh;   // the order of nbr_batch: the same rounding
#pragma unroll
            for (int k = 0; k < D; ++k) {
                hr[k] = -2.f * ri[k];   // exact: a power of two
                b = fmaf(ri[k], ri[k], b);
            }
            hr[D] = -2.f * rh;
            hr[D + 1] = b;
        }
        __syncwarp();
        int cnt = 0;   // list length of home atom h0 + lane (full stencil)

        for (int sr0 = 0; sr0 < Srow; sr0 += 32) {
            // lane: row sr0 + lane of the stencil (offsets of axes 0..D-2),
            // which home atoms reach it, and its pieces along the last axis
            const int sr = sr0 + lane;
            int Jrow = 0;
            uint32_t rcode = 0;
            unsigned amask = 0, mlo = 0, mhi = 0;
            int ps1 = 0, pl1 = 0, ps2 = 0, pl2 = 0, ps3 = 0, pl3 = 0;
            int sgn = 1;   // sign of the row's first non-zero offset (axes 0..D-2; HALF)
            if (sr < Srow) {
                int off[D];
                int rem = sr;
#pragma unroll
                for (int k = D - 2; k >= 0; --k) { off[k] = rem % 3 - 1; rem /= 3; }
                if constexpr (HALF) {
                    sgn = 0;
#pragma unroll
                    for (int k = 0; k < D - 1; ++k) sgn = sgn ? sgn : off[k];
                }
#pragma unroll
                for (int k = 0; k < D - 1; ++k) {
                    int cj = C[k] + off[k];
                    cj = cj < 0 ? cj + n : (cj >= n ? cj - n : cj);
                    Jrow = Jrow * n + cj;
                    rcode |= (uint32_t)(off[k] + 1) << (2 * k);
                }
                Jrow *= n;
                for (int h = 0; h < nh; ++h) {
                    const float *hr = sh + h * HR;
                    float b2 = 0.f;
#pragma unroll
                    for (int k = 0; k < D - 1; ++k) {
                        const float xk = -0.5f * hr[k];
                        float dk = off[k] > 0 ? hLsc - xk : (off[k] < 0 ? xk + hLsc : 0.f);
                        dk = fmaxf(dk, 0.f);
                        b2 = fmaf(dk, dk, b2);
                    }
                    const float reach = (-0.5f * hr[D] + reach_pad) * (1.0f + 1e-5f) + 1e-5f;
                    const float r2 = reach * reach;
                    const float xl = -0.5f * hr[D - 1];
                    const float dlo = fmaxf(xl + hLsc, 0.f), dhi = fmaxf(hLsc - xl, 0.f);
                    if (b2 < r2) amask |= 1u << h;
                    if (fmaf(dlo, dlo, b2) < r2) mlo |= 1u << h;
                    if (fmaf(dhi, dhi, b2) < r2) mhi |= 1u << h;
                }
                if (sgn < 0) amask = 0;   // the mirror half of the stencil (HALF)
                if (amask) {   // a piece no home atom reaches along the last axis is skipped
                    ps1 = dv.cell_start[Jrow + cl_m];
                    pl1 = (mlo && sgn > 0) ? dv.cell_start[Jrow + cl_m + 1] - ps1 : 0;
                    ps2 = dv.cell_start[Jrow + cl];   pl2 = dv.cell_start[Jrow + cl + 1] - ps2;
                    ps3 = dv.cell_start[Jrow + cl_p]; pl3 = mhi ? dv.cell_start[Jrow + cl_p + 1] - ps3 : 0;
                }
            }
            unsigned rows = __ballot_sync(0xffffffffu, amask != 0);
            while (rows) {
                const int src = __ffs(rows) - 1;
                rows &= rows - 1;
                const uint32_t rc0 = __shfl_sync(0xffffffffu, rcode, src);
                const unsigned active = __shfl_sync(0xffffffffu, amask, src);
                const bool zrow = HALF && __shfl_sync(0xffffffffu, sgn, src) == 0;   // offsets 0 on axes 0..D-2
                float offL[D];
#pragma unroll
                for (int k = 0; k < D - 1; ++k) offL[k] = code_offset(rc0, k) * Lsc;
                const int s1 = __shfl_sync(0xffffffffu, ps1, src), l1 = __shfl_sync(0xffffffffu, pl1, src);
                const int s2 = __shfl_sync(0xffffffffu, ps2, src), l2 = __shfl_sync(0xffffffffu, pl2, src);
                const int s3 = __shfl_sync(0xffffffffu, ps3, src), l3 = __shfl_sync(0xffffffffu, pl3, src);
                const int tot = l1 + l2 + l3;
                for (int t0 = 0; t0 < tot; t0 += 32) {
                    const int t = t0 + lane;
                    const bool okj = t < tot;
                    int j, olast;
                    if (t < l1) { j = s1 + t; olast = -1; }
                    else if (t < l1 + l2) { j = s2 + (t - l1); olast = 0; }
                    else { j = s3 + (t - l1 - l2); olast = 1; }
                    if (!okj) { j = s1 < dv.N ? s1 : 0; olast = -1; }
                    float rj[RF];
                    {
                        const float4 *rj4 = reinterpret_cast<const float4 *>(dv.gs0 + (size_t)j * RF);
#pragma unroll
                        for (int q = 0; q < RF / 4; ++q) {
                            const float4 tt = __ldg(rj4 + q);
                            rj[4 * q] = tt.x; rj[4 * q + 1] = tt.y; rj[4 * q + 2] = tt.z; rj[4 * q + 3] = tt.w;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < D - 1; ++k) rj[k] += offL[k];
                    rj[D - 1] = fmaf((float)olast, Lsc, rj[D - 1]);
                    const float rhoj = glob ? dv.hmax_f : rj[D];
                    float Aj = -rhoj * rhoj;
#pragma unroll
                    for (int k = 0; k < D; ++k) Aj = fmaf(rj[k], rj[k], Aj);
                    // |x_j - x_h|^2 - (rho_j + rho_h)^2 for home atom h
                    auto gap = [&](int h) {
                        float hx[HR];
                        const float4 *hr4 = reinterpret_cast<const float4 *>(sh + h * HR);
#pragma unroll
                        for (int q = 0; q < HR / 4; ++q) {
                            const float4 tt = hr4[q];
                            hx[4 * q] = tt.x; hx[4 * q + 1] = tt.y; hx[4 * q + 2] = tt.z; hx[4 * q + 3] = tt.w;
                        }
                        float t = fmaf(rhoj, hx[D], Aj + hx[D + 1]);
#pragma unroll
                        for (int k = 0; k < D; ++k) t = fmaf(rj[k], hx[k], t);
                        return t;
                    };
                    // every reaching home atom, branch-free (warp-uniform loop)
                    unsigned maybe = 0u;
                    for (unsigned act = active; act; act &= act - 1u) {
                        const int h = __ffs(act) - 1;
                        if (gap(h) <= band_x) maybe |= 1u << h;
                    }
                    unsigned keep = okj ? 0xffffffffu : 0u;
                    if constexpr (HALF) {
                        // the home subcell itself: the pairs i < j only
                        if (zrow && olast == 0) {
                            const int dj = j - h0;
                            keep &= dj <= 0 ? 0u : (dj >= 32 ? 0xffffffffu : (1u << dj) - 1u);
                        }
                    } else {
                        if ((unsigned)(j - h0) < (unsigned)nh) keep &= ~(1u << (j - h0));   // not itself
                    }
                    maybe &= keep;
                    unsigned hits = 0u;
                    while (maybe) {   // a hit, or a pair in the band: FP64 decision (x0 at a build)
                        const int h = __ffs(maybe) - 1;
                        maybe &= maybe - 1;
                        if (gap(h) < -band_x) {
                            hits |= 1u << h;
                            continue;
                        }
                        const int i = h0 + h;
                        double s2d = 0.0;
                        for (int k = 0; k < D; ++k) {
                            double dx = dv.x0[(size_t)k * dv.Npad + j] - dv.x0[(size_t)k * dv.Npad + i];
                            dx -= dv.L * rint(dx * dv.invL);
                            s2d += dx * dx;
                        }
                        const double rcd = glob ? dv.rglobal : 0.5 * (dv.sigma[i] + dv.sigma[j]) + dv.skin;
                        if (s2d < rcd * rcd) hits |= 1u << h;
                    }
                    unsigned any = __reduce_or_sync(0xffffffffu, hits);
                    if (!any) continue;
                    const uint32_t wcode = rc0 | ((uint32_t)(olast + 1) << (2 * (D - 1)));
                    if constexpr (HALF) {
                        // the candidate's own list: every home atom it hit (the
                        // opposite offset: 2 - c in every 2-bit field, no borrows),
                        // slots taken by one atomic per candidate (order fixed
                        // afterwards)
                        const uint32_t ncode = (0xAAAAAAAAu & (uint32_t)((1ull << (2 * D)) - 1ull)) - wcode;
                        if (hits) {
                            const int bj = atomicAdd(dv.nnbr + j, __popc(hits));
                            int r = 0;
                            for (unsigned hm = hits; hm; hm &= hm - 1u, ++r) {
                                const int idx = bj + r;
                                if (idx >= dv.cap) break;
                                const int i = h0 + __ffs(hm) - 1;
                                const int64_t pos = list_pos(idx, j, dv.Npad, dv.lgG);
                                if (dv.pack_sh) {
                                    dv.nbr[pos] = (int32_t)pack_entry<D>(dv, i, ncode);
                                } else {
                                    dv.nbr[pos] = i;
                                    dv.code[pos] = ncode;
                                }
                            }
                        }
                    }
                    while (any) {   // home atoms in order; candidates in lane order
                        const int h = __ffs(any) - 1;
                        any &= any - 1u;
                        const bool hit = (hits >> h) & 1u;
                        const unsigned m = __ballot_sync(0xffffffffu, hit);
                        int base;
                        if constexpr (HALF) {   // slots from the list's counter
                            const int lead = __ffs(m) - 1;
                            base = 0;
                            if (lane == lead) base = atomicAdd(dv.nnbr + h0 + h, __popc(m));
                            base = __shfl_sync(0xffffffffu, base, lead);
                        } else {
                            base = __shfl_sync(0xffffffffu, cnt, h);
                        }
                        if (hit) {
                            const int idx = base + __popc(m & ((1u << lane) - 1u));
                            if (idx < dv.cap) {
                                const int64_t pos = list_pos(idx, h0 + h, dv.Npad, dv.lgG);
                                if (dv.pack_sh) {
                                    dv.nbr[pos] = (int32_t)pack_entry<D>(dv, j, wcode);
                                } else {
                                    dv.nbr[pos] = j;
                                    dv.code[pos] = wcode;
                                }
                            }
                        }
                        if (!HALF && lane == h) cnt += __popc(m);
                    }
                }
            }
        }
        if (!HALF && lane < nh) {
            const int i = h0 + lane;
            dv.nnbr[i] = min(cnt, dv.cap);
            if (cnt > dv.cap) atomicOr(&dv.flags->error, (int)ERR_OVERFLOW);
            atomicMax(&dv.flags->max_count, cnt);
            atomicAdd((unsigned long long *)&dv.flags->total_entries, (unsigned long long)cnt);
        }
    }
}

}  // namespace hdmd
