// noalloc.cu -- forces, energy and virial without any device allocation.
//
// Some callers cannot allocate GPU memory at the point where they need
// forces: plug-ins that live inside a host framework whose memory pool owns
// the device, or loops that forbid allocation after start-up (an allocation
// may wait on the whole device).  compute_forces_noalloc serves them: the
// caller passes device
// buffers for the inputs and outputs, and the only other memory the kernel
// touches is the file-scope scratch array below, which the library holds on
// every GPU it is loaded on until the process exits.
//
// The kernel is the FP64 form of the force / energy / virial evaluation with
// the list replaced by all pairs (O(N^2 d) FP64 work), so it needs no Verlet
// list and no cell arrays; its scratch is the per-block partial sums of the
// deterministic energy/virial reduction plus the last-block ticket.  Each
// pair is taken at its nearest image, the only one that can overlap while
// L >= 2 max sigma (the caller's precondition).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/hdmd.h"

namespace {

constexpr int NA_NT = 128;                 // threads (atoms) per block
constexpr int NA_MAX_BLOCKS = 4096;        // => at most 524288 atoms
constexpr int NA_SCRATCH_DOUBLES = 2 * NA_MAX_BLOCKS + 32;

// partial sums: [0, NA_MAX_BLOCKS) energy, [NA_MAX_BLOCKS, 2 NA_MAX_BLOCKS)
// virial, then the ticket counter (an unsigned in the next slot)
static __device__ __align__(256) double g_noalloc_scratch[NA_SCRATCH_DOUBLES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
thread_local std::string g_err;

template <int D>
__global__ void __launch_bounds__(NA_NT) k_forces_allpairs(const double *__restrict__ x,
                                                           const double *__restrict__ sigma,
                                                           int N, double L, double eps,
                                                           double *__restrict__ F,
                                                           double *__restrict__ ew,
                                                           double *__restrict__ scratch) {
    __shared__ double sx[NA_NT * D];
    __shared__ double ss[NA_NT];
    __shared__ double red_e[NA_NT], red_w[NA_NT];
    __shared__ bool last;
    const int i = blockIdx.x * NA_NT + threadIdx.x;
    const bool valid = i < N;
    double xi[D], f[D];
    const double si = valid ? sigma[i] : 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        xi[k] = valid ? x[(size_t)i * D + k] : 0.0;
        f[k] = 0.0;
    }
    const double invL = 1.0 / L;
    double e = 0.0, w = 0.0;
    for (int j0 = 0; j0 < N; j0 += NA_NT) {
        const int jl = j0 + threadIdx.x;
#pragma unroll
        for (int k = 0; k < D; ++k) sx[threadIdx.x * D + k] = jl < N ? x[(size_t)jl * D + k] : 0.0;
        ss[threadIdx.x] = jl < N ? sigma[jl] : 0.0;
        __syncthreads();
        const int nt = min(NA_NT, N - j0);
        if (valid) {
            for (int t = 0; t < nt; ++t) {
                const int j = j0 + t;
                if (j == i) continue;
                double dx[D], r2 = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    double d = xi[k] - sx[t * D + k];
                    d -= L * rint(d * invL);
                    dx[k] = d;
                    r2 += d * d;
                }
                const double s = 0.5 * (si + ss[t]);
                if (r2 < s * s) {
                    const double r = sqrt(r2);
                    const double g = 1.0 - r / s;
                    const double fr = r > 0.0 ? (eps / s) * g / r : 0.0;
#pragma unroll
                    for (int k = 0; k < D; ++k) f[k] += fr * dx[k];
                    e += 0.25 * eps * g * g;   // each pair is seen from both atoms
                    w += 0.5 * fr * r2;
                }
            }
        }
        __syncthreads();
    }
    if (valid) {
#pragma unroll
        for (int k = 0; k < D; ++k) F[(size_t)i * D + k] = f[k];
    }
    // deterministic reduction: block tree, then the last block folds in order
    red_e[threadIdx.x] = e;
    red_w[threadIdx.x] = w;
    __syncthreads();
    for (int s = NA_NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red_e[threadIdx.x] += red_e[threadIdx.x + s];
            red_w[threadIdx.x] += red_w[threadIdx.x + s];
        }
        __syncthreads();
    }
    unsigned *ticket = reinterpret_cast<unsigned *>(scratch + 2 * NA_MAX_BLOCKS);
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = red_e[0];
        scratch[NA_MAX_BLOCKS + blockIdx.x] = red_w[0];
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double E = 0.0, W = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            E += __ldcg(scratch + b);
            W += __ldcg(scratch + NA_MAX_BLOCKS + b);
        }
        ew[0] = E;
        ew[1] = W;
        *ticket = 0u;
    }
}

template <int D>
void launch(int blocks, const double *x, const double *sigma, int N, double L, double eps,
            double *F, double *ew, double *scratch, cudaStream_t s) {
    k_forces_allpairs<D><<<blocks, NA_NT, 0, s>>>(x, sigma, N, L, eps, F, ew, scratch);
}

hdmd_status fail(hdmd_status st, const std::string &m) {
    g_err = m;
    return st;
}

}  // namespace

extern "C" {

const char *hdmd_noalloc_last_error(void) { return g_err.c_str(); }

hdmd_status compute_forces_noalloc(int d, int64_t N, double L, const double *x_dev,
                                   const double *sigma_dev, double eps, double *F_dev,
                                   double *ew_dev, void *cuda_stream) {
    if (d < 2 || d > 10) return fail(HDMD_E_UNSUPPORTED_D, "d must be in 2..10");
    if (N < 2) return fail(HDMD_E_INVALID, "N must be >= 2");
    if (N > (int64_t)NA_MAX_BLOCKS * NA_NT)
        return fail(HDMD_E_INVALID, "N exceeds the scratch limit of compute_forces_noalloc (" +
                                        std::to_string(NA_MAX_BLOCKS * NA_NT) + " atoms)");
    if (!(L > 0.0) || !std::isfinite(L) || !(eps > 0.0) || !std::isfinite(eps))
        return fail(HDMD_E_INVALID, "L and eps must be positive and finite");
    if (!x_dev || !sigma_dev || !F_dev || !ew_dev) return fail(HDMD_E_INVALID, "NULL buffer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HDMD_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(HDMD_E_INVALID, "device index out of range");
    double *scratch;
    {
        // once per device, with that device current: the device address of the array
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return fail(HDMD_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the ticket must start at zero whatever an earlier call left behind
    e = cudaMemsetAsync(scratch + 2 * NA_MAX_BLOCKS, 0, sizeof(double), s);
    if (e != cudaSuccess) return fail(HDMD_E_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int blocks = (int)((N + NA_NT - 1) / NA_NT);
    switch (d) {
        case 2: launch<2>(blocks, x_dev, sigma_dev, (int)N, L, eps, F_dev, ew_dev, scratch, s); break;
        case 3: launch<3>(blocks, x_dev, sigma_dev, (int)N, L, eps, F_dev, ew_dev, scratch, s); break;
        case 4: launch<4>(blocks, x_dev, sigma_dev, (int)N, L, eps, F_dev, ew_dev, scratch, s); break;
        case 5: launch<5>(blocks, x_dev, sigma_dev, (int)N, L, eps, F_dev, ew_dev, scratch, s); break;
        case 6: launch<6>(blocks, x_dev, sigma_dev, (int)N, L, eps, F_dev, ew_dev, scratch, s); break;
        case 7: launch<7>(blocks, x_dev, sigma_dev, (int)N, L, eps, F_dev, ew_dev, scratch, s); break;
        case 8: launch<8>(blocks, x_dev, sigma_dev, (int)N, L, eps, F_dev, ew_dev, scratch, s); break;
        case 9: launch<9>(blocks, x_dev, sigma_dev, (int)N, L, eps, F_dev, ew_dev, scratch, s); break;
        default: launch<10>(blocks, x_dev, sigma_dev, (int)N, L, eps, F_dev, ew_dev, scratch, s); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HDMD_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return HDMD_OK;
}

}  // extern "C"
