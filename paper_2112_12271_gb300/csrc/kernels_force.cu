// kernels_force.cu -- the pair force / energy / virial loop over the full
// Verlet list (Sec. II.B getforce) fused with the velocity-Verlet half kicks
// and drift (Sec. II.B leapfrog, kick-drift-kick), the displacement trigger
// of the list (Sec. II.C) and the FP64 reductions of the thermodynamic and
// FIRE scalars (Sec. II.B FIRE, Sec. II.E getthermo).
//
// Pair law: harmonic soft spheres, U = (eps/2)(1 - r/s_ij)^2 for r < s_ij,
// s_ij = (s_i + s_j)/2, force on i from j = (eps/s_ij)(1 - r/s_ij)(x_i-x_j)/r.
//
// Thread mapping: G consecutive lanes share one atom (G in 1..32); lane g
// walks list entries g, g+G, ... (coalesced thanks to the list layout), the
// partial forces meet through xor shuffles and lane 0 of the group does the
// per-atom epilogue.  FP32 pair arithmetic reads cell-relative FP32 rows
// (x_i - x_j = gs_i - gs_j - o Lsc with o from the entry's code); FP64 pair
// arithmetic reads absolute FP64 rows with the minimum image.  Positions,
// velocities and every global sum stay FP64; sums are reduced per block and
// folded in block order, so results repeat bit for bit.
//
// One MD step of KDK is  kick(F_n) drift -> [rebuild?] -> F_{n+1} kick(F_{n+1}).
// A launch with kick2 + kick1_drift does "F_n; kick(F_n); kick(F_n); drift",
// i.e. the end of step n-1 and the start of step n, reading the gather rows
// of x_n and writing those of x_{n+1} into the other buffer.
#include "launch.h"

namespace hdmd {
namespace {

constexpr int NT = 256;

template <int D, bool FP64P>
__global__ void __launch_bounds__(NT) k_step(Dev dv, StepCfg cfg) {
    constexpr int RF = Rows<D>::RF, RD = Rows<D>::RD;
    __shared__ double sh[(NT / 32) * kNRed];
    const int G = dv.G;
    const int gt = blockIdx.x * NT + threadIdx.x;
    const int i = gt / G;
    const int g = gt - i * G;
    const bool valid = i < dv.N;
    if (cfg.fire_red && dv.flags->fire[FS_STATUS] != (double)FIRE_RUNNING) return;  // loop ended

    double acc[kNRed];
#pragma unroll
    for (int r = 0; r < kNRed; ++r) acc[r] = 0.0;

    double Fi[D];
    double e_i = 0.0, w_i = 0.0;
    if (cfg.compute_force) {
        if (FP64P) {
            double f[D];
#pragma unroll
            for (int k = 0; k < D; ++k) f[k] = 0.0;
            double e = 0.0, w = 0.0;
            if (valid) {
                const double *ri = dv.gd[cfg.in_buf] + (size_t)i * RD;
                double xi[D];
#pragma unroll
                for (int k = 0; k < D; ++k) xi[k] = ri[k];
                const double hi = ri[D];
                const int nn = dv.nnbr[i];
                for (int m = g; m < nn; m += G) {
                    const int j = dv.nbr[list_pos(m, i, dv.Npad, G)];
                    const double *rj = dv.gd[cfg.in_buf] + (size_t)j * RD;
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
                        const double gg = 1.0 - r / s;
                        const double fr = r > 0.0 ? (dv.eps / s) * gg / r : 0.0;
#pragma unroll
                        for (int k = 0; k < D; ++k) f[k] += fr * dx[k];
                        e += 0.5 * dv.eps * gg * gg;
                        w += fr * r2;
                    }
                }
            }
            for (int o = G >> 1; o > 0; o >>= 1) {
#pragma unroll
                for (int k = 0; k < D; ++k) f[k] += __shfl_xor_sync(0xffffffffu, f[k], o);
                e += __shfl_xor_sync(0xffffffffu, e, o);
                w += __shfl_xor_sync(0xffffffffu, w, o);
            }
#pragma unroll
            for (int k = 0; k < D; ++k) Fi[k] = f[k];
            e_i = e;
            w_i = w;
        } else {
            float f[D];
#pragma unroll
            for (int k = 0; k < D; ++k) f[k] = 0.f;
            float e = 0.f, w = 0.f;
            if (valid) {
                const float *ri = dv.gs[cfg.in_buf] + (size_t)i * RF;
                float xi[D];
#pragma unroll
                for (int k = 0; k < D; ++k) xi[k] = ri[k];
                const float hi = ri[D];
                const float Lsc = dv.Lsc_f;
                const float eps = (float)dv.eps;
                const int nn = dv.nnbr[i];
                for (int m = g; m < nn; m += G) {
                    const int64_t pos = list_pos(m, i, dv.Npad, G);
                    const int j = dv.nbr[pos];
                    const uint32_t code = dv.code[pos];
                    const float4 *rj4 = reinterpret_cast<const float4 *>(dv.gs[cfg.in_buf] + (size_t)j * RF);
                    float rj[RF];
#pragma unroll
                    for (int q = 0; q < RF / 4; ++q) {
                        float4 t = __ldg(rj4 + q);
                        rj[4 * q] = t.x; rj[4 * q + 1] = t.y; rj[4 * q + 2] = t.z; rj[4 * q + 3] = t.w;
                    }
                    float dx[D], r2 = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const float o = (float)((int)((code >> (2 * k)) & 3u) - 1);
                        const float t = fmaf(-o, Lsc, xi[k] - rj[k]);
                        dx[k] = t;
                        r2 = fmaf(t, t, r2);
                    }
                    const float s = hi + rj[D];
                    if (r2 < s * s && r2 > 0.f) {
                        const float inv_s = __frcp_rn(s);
                        const float rinv = rsqrtf(r2);
                        const float r = r2 * rinv;
                        const float gg = fmaf(-r, inv_s, 1.f);
                        const float fr = eps * inv_s * gg * rinv;
#pragma unroll
                        for (int k = 0; k < D; ++k) f[k] = fmaf(fr, dx[k], f[k]);
                        e = fmaf(0.5f * eps * gg, gg, e);
                        w = fmaf(fr, r2, w);
                    }
                }
            }
            for (int o = G >> 1; o > 0; o >>= 1) {
#pragma unroll
                for (int k = 0; k < D; ++k) f[k] += __shfl_xor_sync(0xffffffffu, f[k], o);
                e += __shfl_xor_sync(0xffffffffu, e, o);
                w += __shfl_xor_sync(0xffffffffu, w, o);
            }
#pragma unroll
            for (int k = 0; k < D; ++k) Fi[k] = (double)f[k];
            e_i = (double)e;
            w_i = (double)w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) Fi[k] = valid ? dv.F[(size_t)k * dv.Npad + i] : 0.0;
    }

    if (valid && g == 0) {
        const int Np = dv.Npad;
        if (cfg.store_F) {
#pragma unroll
            for (int k = 0; k < D; ++k) dv.F[(size_t)k * Np + i] = Fi[k];
        }
        const double im = dv.inv_mass ? dv.inv_mass[i] : 1.0;
        double v[D];
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = dv.v[(size_t)k * Np + i];
        if (cfg.kick2) {
#pragma unroll
            for (int k = 0; k < D; ++k) v[k] += cfg.halfdt * Fi[k] * im;
        }
        if (cfg.thermo) {
            double v2 = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) v2 += v[k] * v[k];
            acc[R_E] = e_i;
            acc[R_W] = w_i;
            acc[R_K2] = v2 / im;
        }
        if (cfg.fire_red) {
            double P = 0.0, vv = 0.0, vf = 0.0, ff = 0.0, fn = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                P += Fi[k] * v[k];
                vv += v[k] * v[k];
                vf += v[k] * Fi[k] * im;
                ff += (Fi[k] * im) * (Fi[k] * im);
                fn += Fi[k] * Fi[k];
            }
            acc[R_E] = e_i;
            acc[R_P] = P;
            acc[R_VV] = vv;
            acc[R_VF] = vf;
            acc[R_FF] = ff;
            acc[R_FN] = fn;
            acc[R_FMAX2] = fn;
            if (!(fn < INFINITY)) acc[R_BAD] = 1.0;
        }
        if (cfg.kick1_drift) {
            double d2 = 0.0;
            bool bad = false;
            float *go = dv.gs[cfg.out_buf] + (size_t)i * RF;
            const float *g0 = dv.gs0 + (size_t)i * RF;
            double *gdo = dv.gd[cfg.out_buf] + (size_t)i * RD;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                v[k] += cfg.halfdt * Fi[k] * im;
                const size_t o = (size_t)k * Np + i;
                const double dl = dv.dlt[o] + cfg.dt * v[k];
                dv.dlt[o] = dl;
                d2 += dl * dl;
                if (FP64P) gdo[k] = dv.x0[o] + dl;
                else go[k] = g0[k] + (float)dl;
                bad |= !(fabs(dl) < INFINITY) || !(fabs(v[k]) < INFINITY);
            }
            if (FP64P) gdo[D] = 0.5 * dv.sigma[i];
            else go[D] = g0[D];
            acc[R_DMAX2] = d2;
            if (bad) acc[R_BAD] = 1.0;
        }
        if (cfg.kick2 || cfg.kick1_drift) {
#pragma unroll
            for (int k = 0; k < D; ++k) dv.v[(size_t)k * Np + i] = v[k];
        }
    }

    if (cfg.thermo || cfg.fire_red || cfg.kick1_drift) {
        const bool last = block_reduce_and_fold<NT>(dv, acc, R_BAD + 1, dv.maxblocks, sh);
        if (last && threadIdx.x == 0) {
            const double *red = dv.red;
            if (red[R_BAD] != 0.0) atomicOr(&dv.flags->error, (int)ERR_LOST);
            if (cfg.kick1_drift) {
                const double dmax2 = red[R_DMAX2];
                const int trig = (4.0 * dmax2 > dv.skin * dv.skin) || red[R_BAD] != 0.0;
                if (16.0 * dmax2 > dv.L * dv.L) atomicOr(&dv.flags->error, (int)ERR_LOST);
                dv.flags->rebuild = trig;
                if (cfg.cond_rebuild) cudaGraphSetConditional(cfg.cond_rebuild, trig ? 1u : 0u);
            }
            if (cfg.fire_red) {
                // FIRE 2.0 scalar update (Guenole et al. 2020), one thread
                double *fs = dv.flags->fire;
                const double fmx = sqrt(red[R_FMAX2]);
                fs[FS_FMAX] = fmx;
                fs[FS_E] = 0.5 * red[R_E];
                int status = FIRE_RUNNING;
                if (red[R_BAD] != 0.0) status = FIRE_NEGFAIL;
                else if (fmx < fs[FP_FTOL]) status = FIRE_CONVERGED;
                else if (fmx < fs[FP_SWITCH]) status = FIRE_SWITCH;
                else if (fs[FS_ITER] >= fs[FP_MAXITER]) status = FIRE_MAXITER;
                else {
                    double dt = fs[FS_DT], alpha = fs[FS_ALPHA];
                    const double P = red[R_P];
                    if (P > 0.0) {
                        fs[FS_NPOS] += 1.0;
                        fs[FS_NNEG] = 0.0;
                        if (fs[FS_NPOS] > fs[FP_NDELAY]) {
                            dt = fmin(dt * fs[FP_FINC], fs[FP_DTMAX]);
                            alpha *= fs[FP_FALPHA];
                        }
                        fs[FS_BRANCH] = 1.0;
                        // |v + dt F/m| expanded over the sums of this reduction
                        fs[FS_VNORM] = sqrt(fmax(red[R_VV] + 2.0 * dt * red[R_VF] + dt * dt * red[R_FF], 0.0));
                        fs[FS_FNORM] = sqrt(red[R_FN]);
                    } else {
                        fs[FS_NPOS] = 0.0;
                        fs[FS_NNEG] += 1.0;
                        if (fs[FS_NNEG] > fs[FP_NNEGMAX]) status = FIRE_NEGFAIL;
                        if (!(fs[FP_INITDELAY] != 0.0 && fs[FS_ITER] < fs[FP_NDELAY])) {
                            dt = fmax(dt * fs[FP_FDEC], fs[FP_DTMIN]);
                            alpha = fs[FP_ALPHA0];
                        }
                        fs[FS_BRANCH] = 0.0;
                    }
                    fs[FS_DT] = dt;
                    fs[FS_ALPHA] = alpha;
                    if (status == FIRE_RUNNING) {
                        fs[FS_ITER] += 1.0;
                        fs[FS_PHASE_ITER] += 1.0;
                    }
                }
                fs[FS_STATUS] = (double)status;
                if (cfg.cond_loop) cudaGraphSetConditional(cfg.cond_loop, status == FIRE_RUNNING ? 1u : 0u);
            }
        }
    }
}

// FIRE per-atom update, from the scalars the last force reduction left:
//   P <= 0 branch: x -= dt v / 2, v = 0;
//   v += dt F/m;  P > 0 branch: v = (1-alpha) v + alpha |v| F/|F|;  x += dt v.
template <int D>
__global__ void __launch_bounds__(NT) k_fire_update(Dev dv, int write_fp64_rows,
                                                    unsigned long long cond_rebuild) {
    constexpr int RF = Rows<D>::RF, RD = Rows<D>::RD;
    __shared__ double sh[(NT / 32) * kNRed];
    const double *fs = dv.flags->fire;
    if (fs[FS_STATUS] != (double)FIRE_RUNNING) return;
    const double dt = fs[FS_DT], alpha = fs[FS_ALPHA];
    const bool up = fs[FS_BRANCH] != 0.0;
    const double vn = fs[FS_VNORM], fn = fs[FS_FNORM];
    const int i = blockIdx.x * NT + threadIdx.x;
    double acc[kNRed];
#pragma unroll
    for (int r = 0; r < kNRed; ++r) acc[r] = 0.0;
    if (i < dv.N) {
        const int Np = dv.Npad;
        const double im = dv.inv_mass ? dv.inv_mass[i] : 1.0;
        const bool mix = up && fn > 0.0;
        const double cf = mix ? alpha * vn / fn : 0.0;
        double d2 = 0.0;
        bool bad = false;
        float *go = dv.gs[0] + (size_t)i * RF;
        const float *g0 = dv.gs0 + (size_t)i * RF;
        double *gdo = dv.gd[0] + (size_t)i * RD;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const size_t o = (size_t)k * Np + i;
            double v = dv.v[o], dl = dv.dlt[o];
            const double F = dv.F[o];
            if (!up) {
                dl -= 0.5 * dt * v;
                v = 0.0;
            }
            v += dt * F * im;
            if (mix) v = (1.0 - alpha) * v + cf * F;
            dl += dt * v;
            dv.v[o] = v;
            dv.dlt[o] = dl;
            d2 += dl * dl;
            go[k] = g0[k] + (float)dl;
            if (write_fp64_rows) gdo[k] = dv.x0[o] + dl;
            bad |= !(fabs(dl) < INFINITY);
        }
        go[D] = g0[D];
        if (write_fp64_rows) gdo[D] = 0.5 * dv.sigma[i];
        acc[R_DMAX2] = d2;
        if (bad) acc[R_BAD] = 1.0;
    }
    const bool last = block_reduce_and_fold<NT>(dv, acc, R_BAD + 1, dv.maxblocks, sh);
    if (last && threadIdx.x == 0) {
        const double dmax2 = dv.red[R_DMAX2];
        const int trig = (4.0 * dmax2 > dv.skin * dv.skin) || dv.red[R_BAD] != 0.0;
        if (dv.red[R_BAD] != 0.0 || 16.0 * dmax2 > dv.L * dv.L) atomicOr(&dv.flags->error, (int)ERR_LOST);
        dv.flags->rebuild = trig;
        if (cond_rebuild) cudaGraphSetConditional(cond_rebuild, trig ? 1u : 0u);
    }
}

// write gather rows of buffer buf from x0 + dlt (FP32 and/or FP64 rows)
template <int D>
__global__ void k_rows(Dev dv, int buf, int want32, int want64) {
    constexpr int RF = Rows<D>::RF, RD = Rows<D>::RD;
    const int i = blockIdx.x * NT + threadIdx.x;
    if (i >= dv.N) return;
    float *go = dv.gs[buf] + (size_t)i * RF;
    const float *g0 = dv.gs0 + (size_t)i * RF;
    double *gdo = dv.gd[buf] + (size_t)i * RD;
    for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * dv.Npad + i;
        const double dl = dv.dlt[o];
        if (want32) go[k] = g0[k] + (float)dl;
        if (want64) gdo[k] = dv.x0[o] + dl;
    }
    if (want32) go[D] = g0[D];
    if (want64) gdo[D] = 0.5 * dv.sigma[i];
}

template <int D>
void rows_impl(const Dev &dv, int buf, int w32, int w64, cudaStream_t s) {
    k_rows<D><<<(dv.N + NT - 1) / NT, NT, 0, s>>>(dv, buf, w32, w64);
}

template <int D>
void step_impl(const Dev &dv, const StepCfg &cfg, cudaStream_t s) {
    const int64_t threads = (int64_t)dv.N * (cfg.compute_force ? dv.G : 1);
    const int G = cfg.compute_force ? dv.G : 1;
    Dev d2 = dv;
    d2.G = G;   // without a force loop the lanes of a group have nothing to share
    const int blocks = (int)((threads + NT - 1) / NT);
    if (cfg.fp64_pairs)
        k_step<D, true><<<blocks, NT, 0, s>>>(cfg.compute_force ? dv : d2, cfg);
    else
        k_step<D, false><<<blocks, NT, 0, s>>>(cfg.compute_force ? dv : d2, cfg);
}

template <int D>
void fire_update_impl(const Dev &dv, int w64, unsigned long long cond, cudaStream_t s) {
    k_fire_update<D><<<(dv.N + NT - 1) / NT, NT, 0, s>>>(dv, w64, cond);
}

}  // namespace

void launch_step(const Dev &dv, const StepCfg &cfg, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, step_impl, dv, cfg, s);
}

void launch_rows(const Dev &dv, int buf, int want32, int want64, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, rows_impl, dv, buf, want32, want64, s);
}

void launch_fire_update(const Dev &dv, int write_fp64_rows, unsigned long long cond_rebuild,
                        cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, fire_update_impl, dv, write_fp64_rows, cond_rebuild, s);
}

}  // namespace hdmd
