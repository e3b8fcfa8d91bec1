// dev_force.cuh -- the pair force / energy / virial loop over one atom's
// Verlet list, shared by the grid kernels (kernels_force.cu) and the batched
// kernel (kernels_batch.cu).  LAW 0, harmonic spheres: U = (e/2)(1 - r/s)^2
// for r < s = s_ij, force on i = (e/s)(1 - r/s)(x_i - x_j)/r.  LAW 1, the
// truncated and shifted Morse law of Eq. (1): U = e [exp(-2a(r-s)) -
// 2 exp(-a(r-s)) + 1] = e m^2 with m = exp(-a(r-s)) - 1 (evaluated by expm1,
// which keeps its digits near r = s), force on i = 2 a e (m + 1) m
// (x_i - x_j)/r.  e = eps_ij: eps, or with volume-scaled prefactors
// eps (sigma_i sigma_j)^(d/2) = sqrt(eps_i eps_j), eps_i = eps sigma_i^d
// (Sec. II.A), from the radii sigma/2 held in the rows.  LAW 2, the Mie law
// truncated at its minimum s and shifted: U = e [(s/r)^2n - 2 (s/r)^n + 1]
// = e (q - 1)^2 with q = (s/r)^n, force on i = 2 n e (q^2 - q) (x_i - x_j)/r^2.
// Lane g of the atom's group of G = 1 << lgG lanes walks entries g, g+G, ...
// and accumulates its share into f, e (sum of U) and w (sum of r.f); the
// caller combines the lanes.  FP64P selects FP64 pair arithmetic on the
// absolute FP64 rows (minimum image by rint) or FP32 arithmetic on the
// cell-relative FP32 rows with the entry's subcell-offset code.
#pragma once
#include "common.cuh"

#ifndef HDMD_FORCE_UNROLL
#define HDMD_FORCE_UNROLL 3
#endif

namespace hdmd {

// q^n for a small non-negative integer n (binary powering)
template <typename T>
__device__ __forceinline__ T powi(T q, int n) {
    T r = T(1);
    while (n) {
        if (n & 1) r *= q;
        q *= q;
        n >>= 1;
    }
    return r;
}

// pair prefactor from the radii hi, hj: eps, or eps (4 hi hj)^(D/2)
template <int D, typename T>
__device__ __forceinline__ T eps_pair(T eps, T hi, T hj, int scale) {
    if (!scale) return eps;
    const T p = T(4) * hi * hj;
    T q = T(1);
#pragma unroll
    for (int k = 0; k < D / 2; ++k) q *= p;
    if (D & 1) q *= sqrt(p);
    return eps * q;
}

// The pair vector of one list entry in FP32: dx = x_i - x_j - o Lsc (o the
// entry's subcell offsets from its code; x_i - x_j rounds once, the offset
// term is exact and rounds once more), two axes per packed instruction, and
// r2 = |dx|^2 summed in axis order (the bits of the scalar loop)
template <int D>
__device__ __forceinline__ float entry_dx(const float (&xi)[D], const float *rj, uint32_t code, float Lsc,
                                          float (&dx)[D]) {
    const float2 m1 = make_float2(-1.f, -1.f), mL = make_float2(-Lsc, -Lsc);
    const float2 c0 = make_float2(-12582913.0f, -12582913.0f);   // see code_offset
#pragma unroll
    for (int p = 0; p < D / 2; ++p) {
        const float2 ob = make_float2(__uint_as_float(0x4B400000u | ((code >> (4 * p)) & 3u)),
                                      __uint_as_float(0x4B400000u | ((code >> (4 * p + 2)) & 3u)));
        const float2 o = __fadd2_rn(ob, c0);
        const float2 xr = __ffma2_rn(make_float2(rj[2 * p], rj[2 * p + 1]), m1,
                                     make_float2(xi[2 * p], xi[2 * p + 1]));
        const float2 t = __ffma2_rn(o, mL, xr);
        dx[2 * p] = t.x;
        dx[2 * p + 1] = t.y;
    }
    if (D & 1) dx[D - 1] = fmaf(-code_offset(code, D - 1), Lsc, xi[D - 1] - rj[D - 1]);
    float r2 = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) r2 = fmaf(dx[k], dx[k], r2);
    return r2;
}

// One pair's contribution in FP32 arithmetic: dx = x_i - x_j (minimum
// image), r2 = |dx|^2, radii hi, hj (s = hi + hj is the contact distance);
// adds the force on i to f, U to e and r.f to w when r < s.
template <int D, typename FT, int LAW>
__device__ __forceinline__ void pair_term_f32(const Dev &dv, const float (&dx)[D], float r2, float hi,
                                              float hj, float eps, float ma, int scale, FT (&f)[D],
                                              FT &e, FT &w) {
    const float s = hi + hj;
    if (r2 < s * s) {
        // coincident atoms: no force (direction undefined), U(0)
        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
        const float r = r2 * rinv;
        const float ee = eps_pair<D, float>(eps, hi, hj, scale);
        if constexpr (LAW == 2) {
            const float q = powi(s * rinv, dv.mie_n);
            const float fr = 2.f * (float)dv.mie_n * ee * (q * q - q) * rinv * rinv;
#pragma unroll
            for (int k = 0; k < D; ++k) f[k] = (FT)fmaf(fr, dx[k], (float)f[k]);
            e = (FT)fmaf(ee * (q - 1.f), q - 1.f, (float)e);
            w = (FT)fmaf(fr, r2, (float)w);
        } else if constexpr (LAW == 0) {
            const float inv_s = __fdividef(1.f, s);   // approximate: within 2 ulp
            const float gg = fmaf(-r, inv_s, 1.f);
            const float fr = ee * inv_s * gg * rinv;
#pragma unroll
            for (int k = 0; k < D; ++k) f[k] = (FT)fmaf(fr, dx[k], (float)f[k]);
            e = (FT)fmaf(0.5f * ee * gg, gg, (float)e);
            w = (FT)fmaf(fr, r2, (float)w);
        } else {
            const float m = expm1f(-ma * (r - s));
            const float fr = 2.f * ma * ee * (m + 1.f) * m * rinv;
#pragma unroll
            for (int k = 0; k < D; ++k) f[k] = (FT)fmaf(fr, dx[k], (float)f[k]);
            e = (FT)fmaf(ee * m, m, (float)e);
            w = (FT)fmaf(fr, r2, (float)w);
        }
    }
}

// PACK: one-word entries, the offset code looked up in stab (a shared-memory
// table of the 3^D codes by stencil position)
template <int D, bool FP64P, typename FT, int LAW = 0, bool PACK = false>
__device__ __forceinline__ void pair_forces(const Dev &dv, int i, int g, int lgG, int in_buf,
                                            FT (&f)[D], FT &e, FT &w,
                                            const uint32_t *stab = nullptr) {
    constexpr int RF = Rows<D>::RF, RD = Rows<D>::RD;
    const int G = 1 << lgG;
    const int Np = dv.Npad;
    const int nn = HDMD_LDS(dv.nnbr + i);
    if (FP64P) {
        const double *ri = dv.gd[in_buf] + (size_t)i * RD;
        double xi[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xi[k] = ri[k];
        const double hi = ri[D];
        const int64_t lstride = (int64_t)Np << lgG;
        int64_t pos = ((int64_t)i << lgG) + g;
        for (int m = g; m < nn; m += G, pos += lstride) {
            const int j = (int)((uint32_t)dv.nbr[pos] & dv.idx_mask);
            const double *rj = dv.gd[in_buf] + (size_t)j * RD;
            double dx[D], r2 = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                double t = xi[k] - rj[k];
                t -= dv.L * rint(t * dv.invL);
                dx[k] = t;
                r2 += t * t;
            }
            const double s = hi + rj[D];
            if (r2 < s * s) {
                const double r = sqrt(r2);
                const double ee = eps_pair<D, double>(dv.eps, hi, rj[D], dv.eps_scale);
                double fr, u;
                if constexpr (LAW == 0) {
                    const double gg = 1.0 - r / s;
                    fr = r > 0.0 ? (ee / s) * gg / r : 0.0;
                    u = 0.5 * ee * gg * gg;
                } else if constexpr (LAW == 2) {
                    const double q = powi(s / r, dv.mie_n);
                    fr = r > 0.0 ? 2.0 * dv.mie_n * ee * (q * q - q) / r2 : 0.0;
                    u = ee * (q - 1.0) * (q - 1.0);
                } else {
                    const double m = expm1(-dv.morse_a * (r - s));
                    fr = r > 0.0 ? 2.0 * dv.morse_a * ee * (m + 1.0) * m / r : 0.0;
                    u = ee * m * m;
                }
#pragma unroll
                for (int k = 0; k < D; ++k) f[k] += (FT)(fr * dx[k]);
                e += (FT)u;
                w += (FT)(fr * r2);
            }
        }
    } else {
        const float *ri = dv.gs[in_buf] + (size_t)i * RF;
        float xi[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xi[k] = ri[k];
        const float hi = ri[D];
        const float Lsc = dv.Lsc_f;
        const float eps = (float)dv.eps;
        const float ma = (float)dv.morse_a;
        const int scale = dv.eps_scale;
        constexpr int U = HDMD_FORCE_UNROLL;   // list entries in flight per lane
        const int64_t lstride = (int64_t)Np << lgG;
        int64_t pos0 = ((int64_t)i << lgG) + g;
        // the list entries of the next chunk are loaded one chunk ahead (the
        // first chunk before the list length is known: any slot below the
        // capacity may be read; the length decides which entries count).
        // Entries and codes are read once per step: streaming loads, so that
        // they do not push the neighbour rows out of L2.
        const uint32_t *nb = reinterpret_cast<const uint32_t *>(dv.nbr);
        uint32_t jn[U];
        uint32_t cn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool in = g + u * G < dv.cap;
            jn[u] = in ? HDMD_LDS(nb + pos0 + u * lstride) : 0u;
            cn[u] = (!PACK && in) ? HDMD_LDS(dv.code + pos0 + u * lstride) : 0u;
        }
        for (int m0 = g; m0 < nn; m0 += U * G, pos0 += U * lstride) {
            int jv[U];
            uint32_t cv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                jv[u] = m0 + u * G < nn ? (int)(PACK ? jn[u] & dv.idx_mask : jn[u]) : -1;
                cv[u] = PACK ? stab[jv[u] >= 0 ? jn[u] >> dv.pack_sh : 0u] : cn[u];
            }
            if (m0 + U * G < nn) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool ok = m0 + (U + u) * G < nn;
                    const int64_t pos = pos0 + (U + u) * lstride;
                    jn[u] = ok ? HDMD_LDS(nb + pos) : 0u;
                    cn[u] = (!PACK && ok) ? HDMD_LDS(dv.code + pos) : 0u;
                }
            }
            float rj[U][RF];
#pragma unroll
            for (int u = 0; u < U; ++u)
                load_row<RF, true>(dv.gs[in_buf] + (size_t)(jv[u] >= 0 ? jv[u] : i) * RF, rj[u]);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (jv[u] < 0) continue;
                float dx[D];
                const float r2 = entry_dx<D>(xi, rj[u], cv[u], Lsc, dx);
                pair_term_f32<D, FT, LAW>(dv, dx, r2, hi, rj[u][D], eps, ma, scale, f, e, w);
            }
        }
    }
}

}  // namespace hdmd
