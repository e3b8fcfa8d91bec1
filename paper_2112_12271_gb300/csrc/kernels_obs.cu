// kernels_obs.cu -- the Berendsen barostat's rescaling of the positions and
// the on-device observables of Sec. II.E: mean squared and
// quartic displacements since a reference configuration, the non-Gaussian
// parameter alpha_2 (Eq. (14)), the overlap function f_ov (Eq. (15)), the
// self part of the van Hove function G_s(r, t) (Eq. (16)) as a histogram,
// and the mean coordination number Z (interacting neighbours, r < sigma_ij).
//
// Displacements use unwrapped FP64 positions x0 + dlt + L img against the
// reference stored in caller order (row-major [N][d]); the internal slot s
// holds caller atom id[s].  Sums are reduced per block and folded in block
// order (bitwise repeatable); the histogram and Z are integer counts.
#include "launch.h"

namespace hdmd {
namespace {

constexpr int NT = 256;
inline int nblk(int n) { return (n + NT - 1) / NT; }

template <int D>
__global__ void k_ref_from_current(Dev dv, double *ref) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= dv.N) return;
    const int c = dv.id[s];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * dv.Npad + s;
        ref[(size_t)c * D + k] = dv.x0[o] + dv.dlt[o] + dv.L * (double)dv.img[o];
    }
}

template <int D>
__global__ void __launch_bounds__(NT) k_observe(Dev dv, const double *ref, double a2, int nbins,
                                                double inv_w, unsigned int *hist, int want_z) {
    __shared__ double sh[(NT / 32) * kNRed];
    double acc[kNRed];
#pragma unroll
    for (int r = 0; r < kNRed; ++r) acc[r] = 0.0;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < dv.N) {
        const int c = dv.id[s];
        double dr2 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const size_t o = (size_t)k * dv.Npad + s;
            const double t = dv.x0[o] + dv.dlt[o] + dv.L * (double)dv.img[o] - ref[(size_t)c * D + k];
            dr2 += t * t;
        }
        acc[0] = dr2;              // MSD
        acc[1] = dr2 * dr2;        // MQD
        acc[2] = dr2 < a2 ? 1.0 : 0.0;   // f_ov
        if (nbins > 0) {
            const double b = sqrt(dr2) * inv_w;
            if (b < (double)nbins) atomicAdd(hist + (int)b, 1u);
        }
        if (want_z) {              // neighbours closer than sigma_ij, over the list
            const int nn = dv.nnbr[s];
            int z = 0;
            for (int m = 0; m < nn; ++m) {
                const int j = (int)((uint32_t)dv.nbr[list_pos(m, s, dv.Npad, dv.lgG)] & dv.idx_mask);
                double r2 = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const size_t oi = (size_t)k * dv.Npad + s, oj = (size_t)k * dv.Npad + j;
                    double t = (dv.x0[oj] + dv.dlt[oj]) - (dv.x0[oi] + dv.dlt[oi]);
                    t -= dv.L * rint(t * dv.invL);
                    r2 += t * t;
                }
                const double sij = 0.5 * (dv.sigma[s] + dv.sigma[j]);
                z += r2 < sij * sij;
            }
            acc[R_P] = (double)z;   // slot 4 (a sum slot)
        }
    }
    block_reduce_and_fold<NT>(dv, acc, R_P + 1, dv.maxblocks, sh);
}

// Berendsen barostat: every position (x0 + dlt, the box centred at the
// origin) is multiplied by mu; the displacement since the build is folded
// into x0 (the list build that follows wraps and rebins)
template <int D>
__global__ void k_scale_positions(Dev dv, double mu) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= dv.N) return;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const size_t o = (size_t)k * dv.Npad + s;
        dv.x0[o] = mu * (dv.x0[o] + dv.dlt[o]);
        dv.dlt[o] = 0.0;
    }
}

template <int D> void scale_impl(const Dev &dv, double mu, cudaStream_t s) {
    k_scale_positions<D><<<nblk(dv.N), NT, 0, s>>>(dv, mu);
}

template <int D> void ref_impl(const Dev &dv, double *ref, cudaStream_t s) {
    k_ref_from_current<D><<<nblk(dv.N), NT, 0, s>>>(dv, ref);
}
template <int D> void observe_impl(const Dev &dv, const double *ref, double a2, int nbins,
                                   double inv_w, unsigned int *hist, int want_z, cudaStream_t s) {
    k_observe<D><<<nblk(dv.N), NT, 0, s>>>(dv, ref, a2, nbins, inv_w, hist, want_z);
}

}  // namespace

void launch_scale_positions(const Dev &dv, double mu, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, scale_impl, dv, mu, s);
}
void launch_reference(const Dev &dv, double *ref, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, ref_impl, dv, ref, s);
}
void launch_observe(const Dev &dv, const double *ref, double a2, int nbins, double inv_w,
                    unsigned int *hist, int want_z, cudaStream_t s) {
    HDMD_DISPATCH_D(dv.d, observe_impl, dv, ref, a2, nbins, inv_w, hist, want_z, s);
}

}  // namespace hdmd
