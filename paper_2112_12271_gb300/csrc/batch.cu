// batch.cu -- host side of the batched engine (C ABI batch_* in hdmd.h).
//
// A batch owns one device pool.  Each job (an MD run or a FIRE minimisation
// of its own N, d, L and diameters) is carved out of the pool by a first-fit
// allocator when it is admitted; a job that does not fit is refused
// (HDMD_E_NOMEM) so the caller can admit it later, when finished jobs have
// been removed (admission by free device memory).  batch_run launches one
// persistent kernel per dimension present, side by side on forked streams,
// captured once into a CUDA graph; each kernel's blocks take the jobs of its
// dimension from a device queue, largest first.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/hdmd.h"
#include "batch.cuh"
#include "launch.h"

using namespace hdmd;

namespace {

thread_local std::string g_batch_err;

struct Pool {
    size_t bytes = 0;
    std::map<size_t, size_t> free_;   // offset -> size
    void init(size_t b) { bytes = b; free_.clear(); free_[0] = b; }
    // first fit, 256-byte aligned sizes
    long long alloc(size_t size) {
        size = (size + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= size) {
                size_t off = it->first, rest = it->second - size;
                free_.erase(it);
                if (rest) free_[off + size] = rest;
                return (long long)off;
            }
        }
        return -1;
    }
    void release(size_t off, size_t size) {
        size = (size + 255) & ~(size_t)255;
        auto it = free_.emplace(off, size).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t free_bytes() const {
        size_t s = 0;
        for (auto &kv : free_) s += kv.second;
        return s;
    }
};

struct HostJob {
    bool live = false;
    int d = 0;
    int64_t N = 0;
    size_t off = 0, size = 0;
    int cap = 0;
};

// Lay out the arrays of one job from base (or only count bytes when base is
// NULL).  Returns the bytes used.
size_t layout(Dev &dv, char *base, int cap) {
    size_t off = 0;
    const size_t Np = dv.Npad, nd = (size_t)dv.d * Np;
    const int RF = kRowFloats(dv.d), RD = kRowDoubles(dv.d);
    auto take = [&](auto *&ptr, size_t count) {
        using T = typename std::remove_reference<decltype(*ptr)>::type;
        off = (off + 255) & ~(size_t)255;
        if (base) ptr = reinterpret_cast<T *>(base + off);
        off += sizeof(T) * (count ? count : 1);
    };
    take(dv.x0, nd); take(dv.dlt, nd); take(dv.v, nd); take(dv.F, nd);
    take(dv.sigma, Np);
    take(dv.img, nd); take(dv.id, Np);
    take(dv.gs0, Np * RF); take(dv.gs[0], Np * RF);
    take(dv.gd[0], Np * RD);
    take(dv.cell_count, dv.ncells); take(dv.cell_fill, dv.ncells);
    take(dv.cell_start, dv.ncells + 1); take(dv.batch_start, dv.ncells + 1);
    take(dv.cell_of, Np); take(dv.perm, Np); take(dv.cellid, Np);
    take(dv.tx, nd); take(dv.tv, nd); take(dv.tsig, Np); take(dv.tim, Np);
    take(dv.timg, nd); take(dv.tid, Np);
    take(dv.nnbr, Np);
    take(dv.nbr, (size_t)cap * Np);
    take(dv.code, (size_t)cap * Np);
    take(dv.flags, 1);
    if (base) {
        dv.gs[1] = dv.gs[0];
        dv.gd[1] = dv.gd[0];
        dv.inv_mass = nullptr;
        dv.partials = nullptr;
        dv.red = nullptr;
    }
    return off;
}

}  // namespace

struct hdmd_batch {
    cudaStream_t stream = nullptr;
    cudaStream_t fork[2 * (kMaxD + 1)] = {nullptr};       // [d]: normal, [kMaxD + 1 + d]: wide
    cudaEvent_t ev_fork = nullptr, ev_join[2 * (kMaxD + 1)] = {nullptr};
    int prec = HDMD_MIXED;
    char *pool_dev = nullptr;
    Pool pool;
    int max_jobs = 0;
    BatchJob *d_jobs = nullptr, *h_jobs = nullptr;
    int *d_order = nullptr, *h_order = nullptr;
    BatchCtl *d_ctl = nullptr, *h_ctl = nullptr;
    std::vector<HostJob> jobs;
    int lgG[kMaxD + 1];
    int nsm = 152;
    std::map<unsigned, std::pair<cudaGraph_t, cudaGraphExec_t>> graphs;   // dims bitmask
    bool use_graphs = true;
    std::string err;
};

namespace {

hdmd_status bfail(hdmd_batch *b, hdmd_status st, const std::string &m) {
    g_batch_err = m;
    if (b) b->err = m;
    return st;
}

#define BCK(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return bfail(b, HDMD_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void launch_one(int d, BatchJob *jobs, const int *order, BatchCtl *ctl, int grid, cudaStream_t s) {
    switch (d) {
        case 2: launch_batch_d2(jobs, order, ctl, grid, s); break;
        case 3: launch_batch_d3(jobs, order, ctl, grid, s); break;
        case 4: launch_batch_d4(jobs, order, ctl, grid, s); break;
        case 5: launch_batch_d5(jobs, order, ctl, grid, s); break;
        case 6: launch_batch_d6(jobs, order, ctl, grid, s); break;
        case 7: launch_batch_d7(jobs, order, ctl, grid, s); break;
        case 8: launch_batch_d8(jobs, order, ctl, grid, s); break;
        case 9: launch_batch_d9(jobs, order, ctl, grid, s); break;
        case 10: launch_batch_d10(jobs, order, ctl, grid, s); break;
        default: break;
    }
}

void launch_one_wide(int d, BatchJob *jobs, const int *order, BatchCtl *ctl, int grid,
                     cudaStream_t s) {
    switch (d) {
        case 2: launch_batch_wide_d2(jobs, order, ctl, grid, s); break;
        case 3: launch_batch_wide_d3(jobs, order, ctl, grid, s); break;
        case 4: launch_batch_wide_d4(jobs, order, ctl, grid, s); break;
        case 5: launch_batch_wide_d5(jobs, order, ctl, grid, s); break;
        case 6: launch_batch_wide_d6(jobs, order, ctl, grid, s); break;
        case 7: launch_batch_wide_d7(jobs, order, ctl, grid, s); break;
        case 8: launch_batch_wide_d8(jobs, order, ctl, grid, s); break;
        case 9: launch_batch_wide_d9(jobs, order, ctl, grid, s); break;
        case 10: launch_batch_wide_d10(jobs, order, ctl, grid, s); break;
        default: break;
    }
}

void probe_one(int d, BatchJob *job, int reps, cudaStream_t s) {
    switch (d) {
        case 2: launch_batch_probe_d2(job, reps, s); break;
        case 3: launch_batch_probe_d3(job, reps, s); break;
        case 4: launch_batch_probe_d4(job, reps, s); break;
        case 5: launch_batch_probe_d5(job, reps, s); break;
        case 6: launch_batch_probe_d6(job, reps, s); break;
        case 7: launch_batch_probe_d7(job, reps, s); break;
        case 8: launch_batch_probe_d8(job, reps, s); break;
        case 9: launch_batch_probe_d9(job, reps, s); break;
        case 10: launch_batch_probe_d10(job, reps, s); break;
        default: break;
    }
}

// grid of each per-dimension kernel: two blocks per SM (its occupancy), so a
// launch of every dimension fills the GPU however the jobs are split
int grid_for(const hdmd_batch *b) { return 2 * b->nsm; }

}  // namespace

extern "C" {

const char *hdmd_batch_last_error(const hdmd_batch *b) {
    return b ? b->err.c_str() : g_batch_err.c_str();
}

hdmd_status batch_create(int64_t pool_bytes, int max_jobs, hdmd_precision prec, void *cuda_stream,
                         hdmd_batch **out) {
    hdmd_batch *b = nullptr;
    if (!out) return bfail(nullptr, HDMD_E_INVALID, "out is NULL");
    *out = nullptr;
    if (pool_bytes < (1 << 20) || max_jobs < 1 || max_jobs > (1 << 20))
        return bfail(nullptr, HDMD_E_INVALID, "pool_bytes >= 1 MiB and 1 <= max_jobs <= 2^20 required");
    if (prec != HDMD_FP64 && prec != HDMD_MIXED) return bfail(nullptr, HDMD_E_INVALID, "unknown precision");
    b = new hdmd_batch();
    b->stream = (cudaStream_t)cuda_stream;
    b->prec = prec;
    b->max_jobs = max_jobs;
    b->jobs.resize(max_jobs);
    for (int d = 0; d <= kMaxD; ++d) b->lgG[d] = 2;   // 4 lanes per atom until tuned
    auto bail = [&](hdmd_status st) { batch_destroy(b); return st; };
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    if (cudaMalloc((void **)&b->pool_dev, (size_t)pool_bytes) != cudaSuccess) {
        cudaGetLastError();
        return bail(bfail(b, HDMD_E_NOMEM, "batch pool allocation failed"));
    }
    b->pool.init((size_t)pool_bytes);
    if (cudaMalloc((void **)&b->d_jobs, sizeof(BatchJob) * max_jobs) != cudaSuccess ||
        cudaMalloc((void **)&b->d_order, sizeof(int) * max_jobs) != cudaSuccess ||
        cudaMalloc((void **)&b->d_ctl, sizeof(BatchCtl) * 2 * (kMaxD + 1)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_jobs, sizeof(BatchJob) * max_jobs) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_order, sizeof(int) * max_jobs) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_ctl, sizeof(BatchCtl) * 2 * (kMaxD + 1)) != cudaSuccess) {
        cudaGetLastError();
        return bail(bfail(b, HDMD_E_NOMEM, "batch tables"));
    }
    std::memset(b->h_jobs, 0, sizeof(BatchJob) * max_jobs);
    if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return bail(bfail(b, HDMD_E_CUDA, "event"));
    for (int k = 0; k < 2 * (kMaxD + 1); ++k) {
        if (k % (kMaxD + 1) < 2) continue;
        if (cudaStreamCreateWithFlags(&b->fork[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return bail(bfail(b, HDMD_E_CUDA, "streams"));
        }
    }
    *out = b;
    return HDMD_OK;
}

hdmd_status batch_add(hdmd_batch *b, const hdmd_job_spec *spec, const double *diameters,
                      const double *x, const double *v, int *job_id) {
    if (!b) return bfail(nullptr, HDMD_E_INVALID, "null batch");
    if (!spec || !diameters || !x || !job_id) return bfail(b, HDMD_E_INVALID, "NULL argument");
    const int d = spec->d;
    const int64_t N = spec->N;
    if (d < 2 || d > kMaxD) return bfail(b, HDMD_E_UNSUPPORTED_D, "d must be in 2..10");
    if (N < 2 || N > (1 << 24)) return bfail(b, HDMD_E_INVALID, "N must be in 2..2^24");
    if (spec->kind != 0 && spec->kind != 1) return bfail(b, HDMD_E_INVALID, "kind must be 0 (MD) or 1 (FIRE)");
    if (!(spec->L > 0) || !(spec->eps > 0) || !(spec->skin >= 0) || !std::isfinite(spec->L))
        return bfail(b, HDMD_E_INVALID, "L, eps must be positive and skin >= 0");
    if (spec->kind == 0 && (!(spec->dt > 0) || spec->nsteps < 0))
        return bfail(b, HDMD_E_INVALID, "MD jobs need dt > 0 and nsteps >= 0");
    double smax = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (!(diameters[i] > 0) || !std::isfinite(diameters[i]))
            return bfail(b, HDMD_E_INVALID, "diameters must be positive and finite");
        smax = std::max(smax, diameters[i]);
    }
    for (int64_t a = 0; a < N * d; ++a)
        if (!std::isfinite(x[a]) || (v && !std::isfinite(v[a])))
            return bfail(b, HDMD_E_INVALID, "non-finite position or velocity");
    if (!(spec->L > 2.0 * smax))
        return bfail(b, HDMD_E_INVALID, "box too small: L must exceed twice the largest diameter");
    if (spec->kind != 0 && spec->fire.dt0 > 0 && spec->fire.dx_max != 0.0)
        return bfail(b, HDMD_E_INVALID, "dx_max is not available in the batched engine");
    int n = std::max(1, (int)std::floor(spec->L / (smax + spec->skin)));   // Eq. (7)
    while (n > 2 && std::pow((double)n, d) > 8.0 * (double)N + 4096.0) --n;
    int id = -1;
    for (int k = 0; k < b->max_jobs; ++k)
        if (!b->jobs[k].live) { id = k; break; }
    if (id < 0) return bfail(b, HDMD_E_NOMEM, "all job slots are in use");

    Dev dv;
    std::memset(&dv, 0, sizeof(dv));
    dv.d = d;
    dv.N = (int)N;
    dv.Npad = (int)((N + 63) / 64 * 64);
    dv.G = 1 << b->lgG[d];
    dv.lgG = b->lgG[d];
    dv.idx_mask = 0xFFFFFFFFu;   // jobs keep the index and code arrays
    dv.pack_sh = 0;
    dv.L = spec->L;
    dv.halfL = 0.5 * spec->L;
    dv.invL = 1.0 / spec->L;
    dv.skin = spec->skin;
    dv.eps = spec->eps;
    dv.n = n;
    dv.ncells = 1;
    for (int k = 0; k < d; ++k) dv.ncells *= n;
    dv.Lsc = spec->L / n;
    dv.invLsc = n / spec->L;
    dv.Lsc_f = (float)dv.Lsc;
    dv.L_f = (float)spec->L;
    dv.halfL_f = (float)(0.5 * spec->L);
    dv.hmax_f = (float)(0.5 * smax);
    const double rho = (double)N / std::pow(spec->L, d);
    const double R = smax + spec->skin;
    const double vball = std::pow(M_PI, 0.5 * d) * std::pow(R, d) / std::tgamma(1.0 + 0.5 * d);
    int cap = spec->list_capacity > 0 ? spec->list_capacity
                                      : (int)std::min(2.0 * rho * vball + 24.0, (double)N + 8.0);
    cap = (cap + 31) / 32 * 32;   // a multiple of every lanes-per-atom choice
    dv.cap = cap;
    const size_t bytes = layout(dv, nullptr, cap);
    const long long off = b->pool.alloc(bytes);
    if (off < 0)
        return bfail(b, HDMD_E_NOMEM, "the batch pool has no room for this job now (" +
                                          std::to_string(bytes) + " bytes)");
    layout(dv, b->pool_dev + off, cap);
    HostJob &hj = b->jobs[id];
    hj.live = true;
    hj.d = d;
    hj.N = N;
    hj.off = (size_t)off;
    hj.size = bytes;
    hj.cap = cap;
    // initial state: SoA positions and velocities, identity order
    const size_t Np = dv.Npad;
    std::vector<double> xs((size_t)d * Np, 0.0), vs((size_t)d * Np, 0.0), sg(Np, 1.0);
    std::vector<int32_t> ids(Np);
    for (int64_t i = 0; i < N; ++i) {
        for (int k = 0; k < d; ++k) {
            xs[(size_t)k * Np + i] = x[i * d + k];
            if (v) vs[(size_t)k * Np + i] = v[i * d + k];
        }
        sg[i] = diameters[i];
    }
    for (size_t i = 0; i < Np; ++i) ids[i] = (int32_t)i;
    cudaStream_t s = b->stream;
    hdmd_status st = HDMD_OK;
    auto fail_free = [&](const char *what, cudaError_t e) {
        cudaGetLastError();
        b->pool.release(hj.off, hj.size);
        hj.live = false;
        return bfail(b, HDMD_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMemsetAsync(b->pool_dev + off, 0, bytes, s)) != cudaSuccess) return fail_free("memset", e);
    if ((e = cudaMemcpyAsync(dv.x0, xs.data(), sizeof(double) * xs.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dv.v, vs.data(), sizeof(double) * vs.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dv.sigma, sg.data(), sizeof(double) * Np, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dv.id, ids.data(), sizeof(int32_t) * Np, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail_free("upload", e);
    BatchJob &J = b->h_jobs[id];
    std::memset(&J, 0, sizeof(J));
    J.dv = dv;
    J.kind = spec->kind == 0 ? JOB_MD : JOB_FIRE;
    J.status = JOB_ACTIVE;
    J.mixed = b->prec == HDMD_MIXED;
    J.phase64 = b->prec == HDMD_FP64;
    J.lgG = b->lgG[d];
    J.nsteps = spec->nsteps;
    J.dt = spec->dt;
    if (J.kind == JOB_FIRE) {
        hdmd_fire_params p = spec->fire;
        if (!(p.dt0 > 0)) {
            p.e_thres = 0.0; p.f_thres = 0.0; p.dx_max = 0.0;
            p.dt0 = 0.005; p.dt_max = 0.05; p.dt_min = 1e-4; p.f_inc = 1.1; p.f_dec = 0.5;
            p.alpha0 = 0.25; p.f_alpha = 0.99; p.f_tol = 1e-10; p.polish_tol = 1e-6;
            p.n_delay = 20; p.n_neg_max = 2000; p.max_iter = 1000000; p.initial_delay = 1;
        }
        double *fs = J.fire;
        fs[FS_DT] = p.dt0;
        fs[FS_ALPHA] = p.alpha0;
        fs[FS_STATUS] = FIRE_RUNNING;
        fs[FP_DTMAX] = p.dt_max;
        fs[FP_DTMIN] = p.dt_min;
        fs[FP_FINC] = p.f_inc;
        fs[FP_FDEC] = p.f_dec;
        fs[FP_ALPHA0] = p.alpha0;
        fs[FP_FALPHA] = p.f_alpha;
        fs[FP_FTOL] = p.f_tol;
        fs[FP_SWITCH] = (J.mixed && p.polish_tol > p.f_tol) ? p.polish_tol : 0.0;
        fs[FP_NDELAY] = (double)p.n_delay;
        fs[FP_NNEGMAX] = (double)p.n_neg_max;
        fs[FP_MAXITER] = (double)p.max_iter;
        fs[FP_INITDELAY] = p.initial_delay ? 1.0 : 0.0;
        fs[FP_ETHRES] = p.e_thres;
        fs[FP_FTHRES] = p.f_thres;
        fs[FP_DXMAX] = 0.0;
        fs[FP_NATOMS] = (double)N;
        fs[FS_FITER] = -1.0;
    }
    if ((e = cudaMemcpyAsync(b->d_jobs + id, &J, sizeof(J), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail_free("descriptor", e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_free("sync", e);
    *job_id = id;
    return st;
}

hdmd_status batch_run(hdmd_batch *b, int64_t budget, int *n_unfinished) {
    if (!b) return bfail(nullptr, HDMD_E_INVALID, "null batch");
    if (budget < 0) return bfail(b, HDMD_E_INVALID, "budget must be >= 0");
    // queues per dimension, largest job first
    // (the jobs above kBatchWideN atoms, at the head of each queue, run in the
    // wide blocks of their own kernel: ctl[kMaxD + 1 + d])
    std::vector<std::vector<int>> per(kMaxD + 1);
    for (int k = 0; k < b->max_jobs; ++k)
        if (b->jobs[k].live && b->h_jobs[k].status == JOB_ACTIVE) per[b->jobs[k].d].push_back(k);
    unsigned dims = 0, wdims = 0;
    int pos = 0;
    for (int d = 2; d <= kMaxD; ++d) {
        auto &q = per[d];
        std::stable_sort(q.begin(), q.end(), [&](int a, int c) { return b->jobs[a].N > b->jobs[c].N; });
        int nw = 0;
        while (nw < (int)q.size() && b->jobs[q[nw]].N > kBatchWideN) ++nw;
        BatchCtl &cw = b->h_ctl[kMaxD + 1 + d], &cn = b->h_ctl[d];
        cw.first = pos;
        cw.njobs = nw;
        cw.next = 0;
        cw.budget = budget;
        cn.first = pos + nw;
        cn.njobs = (int)q.size() - nw;
        cn.next = 0;
        cn.budget = budget;
        for (size_t k = 0; k < q.size(); ++k) b->h_order[pos + k] = q[k];
        if (cn.njobs > 0) dims |= 1u << d;
        if (nw > 0) wdims |= 1u << d;
        pos += (int)q.size();
    }
    if (!dims && !wdims) {
        if (n_unfinished) *n_unfinished = 0;
        return HDMD_OK;
    }
    cudaStream_t s = b->stream;
    BCK(cudaMemcpyAsync(b->d_order, b->h_order, sizeof(int) * std::max(pos, 1), cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(b->d_ctl, b->h_ctl, sizeof(BatchCtl) * 2 * (kMaxD + 1), cudaMemcpyHostToDevice, s));
    auto run_direct = [&]() -> hdmd_status {
        BCK(cudaEventRecord(b->ev_fork, s));
        for (int k = 0; k < 2 * (kMaxD + 1); ++k) {
            const bool wide = k > kMaxD;
            const int d = wide ? k - (kMaxD + 1) : k;
            if (d < 2 || !((wide ? wdims : dims) & (1u << d))) continue;
            BCK(cudaStreamWaitEvent(b->fork[k], b->ev_fork, 0));
            if (wide) launch_one_wide(d, b->d_jobs, b->d_order, b->d_ctl + k, b->nsm, b->fork[k]);
            else launch_one(d, b->d_jobs, b->d_order, b->d_ctl + k, grid_for(b), b->fork[k]);
            BCK(cudaGetLastError());
            BCK(cudaEventRecord(b->ev_join[k], b->fork[k]));
            BCK(cudaStreamWaitEvent(s, b->ev_join[k], 0));
        }
        return HDMD_OK;
    };
    hdmd_status st = HDMD_OK;
    // kernel arguments depend only on which dimensions (and block classes) run
    const unsigned key = dims | (wdims << 16);
    bool launched = false;
    if (b->use_graphs) {
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaStream_t cs = nullptr;
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ex = nullptr;
            bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) == cudaSuccess;
            if (ok) {
                cudaStream_t keep = s;
                s = cs;
                st = run_direct();
                s = keep;
                ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && st == HDMD_OK &&
                     cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
            }
            if (cs) cudaStreamDestroy(cs);
            cudaGetLastError();
            if (ok) {
                it = b->graphs.emplace(key, std::make_pair(g, ex)).first;
            } else {
                if (g) cudaGraphDestroy(g);
                b->use_graphs = false;
                st = HDMD_OK;
            }
        }
        if (b->use_graphs) {
            BCK(cudaGraphLaunch(it->second.second, s));
            launched = true;
        }
    }
    if (!launched) {
        st = run_direct();
        if (st) return st;
    }
    // read every descriptor back
    int hi = 0;
    for (int k = 0; k < b->max_jobs; ++k) if (b->jobs[k].live) hi = k + 1;
    BCK(cudaMemcpyAsync(b->h_jobs, b->d_jobs, sizeof(BatchJob) * std::max(hi, 1), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    int left = 0;
    for (int k = 0; k < hi; ++k)
        if (b->jobs[k].live && b->h_jobs[k].status == JOB_ACTIVE) ++left;
    if (n_unfinished) *n_unfinished = left;
    return HDMD_OK;
}

hdmd_status batch_result(hdmd_batch *b, int job_id, hdmd_job_result *res, double *x) {
    if (!b) return bfail(nullptr, HDMD_E_INVALID, "null batch");
    if (job_id < 0 || job_id >= b->max_jobs || !b->jobs[job_id].live)
        return bfail(b, HDMD_E_INVALID, "no such job");
    const BatchJob &J = b->h_jobs[job_id];
    if (res) {
        res->status = J.status;
        res->kind = J.kind;
        res->iterations = J.kind == JOB_FIRE ? (int64_t)J.fire[FS_ITER] : J.steps_done;
        res->rebuilds = J.builds;
        res->E_pair = 0.5 * J.sums[R_E];
        res->virial = 0.5 * J.sums[R_W];
        res->K = 0.5 * J.sums[R_K2];
        res->fmax = std::sqrt(J.sums[R_FMAX2]);
        res->converged = J.kind == JOB_FIRE && J.status == JOB_DONE;
        res->error = J.error;
    }
    if (x) {
        const Dev &dv = J.dv;
        const size_t Np = dv.Npad, nd = (size_t)dv.d * Np;
        std::vector<double> x0(nd), dl(nd);
        std::vector<int32_t> id(Np);
        cudaStream_t s = b->stream;
        BCK(cudaMemcpyAsync(x0.data(), dv.x0, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
        BCK(cudaMemcpyAsync(dl.data(), dv.dlt, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
        BCK(cudaMemcpyAsync(id.data(), dv.id, sizeof(int32_t) * Np, cudaMemcpyDeviceToHost, s));
        BCK(cudaStreamSynchronize(s));
        for (int i = 0; i < dv.N; ++i) {
            for (int k = 0; k < dv.d; ++k) {
                double p = x0[(size_t)k * Np + i] + dl[(size_t)k * Np + i];
                p -= dv.L * std::floor((p + dv.halfL) * dv.invL);
                if (p >= dv.halfL) p -= dv.L;
                if (p < -dv.halfL) p += dv.L;
                x[(size_t)id[i] * dv.d + k] = p;
            }
        }
    }
    return HDMD_OK;
}

hdmd_status batch_remove(hdmd_batch *b, int job_id) {
    if (!b) return bfail(nullptr, HDMD_E_INVALID, "null batch");
    if (job_id < 0 || job_id >= b->max_jobs || !b->jobs[job_id].live)
        return bfail(b, HDMD_E_INVALID, "no such job");
    HostJob &hj = b->jobs[job_id];
    b->pool.release(hj.off, hj.size);
    hj.live = false;
    b->h_jobs[job_id].status = JOB_DONE;
    return HDMD_OK;
}

hdmd_status batch_info(hdmd_batch *b, int64_t *free_bytes, int *live_jobs, int *lanes_by_d) {
    if (!b) return bfail(nullptr, HDMD_E_INVALID, "null batch");
    if (free_bytes) *free_bytes = (int64_t)b->pool.free_bytes();
    if (live_jobs) {
        int c = 0;
        for (auto &j : b->jobs) c += j.live;
        *live_jobs = c;
    }
    if (lanes_by_d)
        for (int d = 0; d <= kMaxD; ++d) lanes_by_d[d] = 1 << b->lgG[d];
    return HDMD_OK;
}

// Lanes-per-atom autotuner: for every dimension with live jobs, time the
// force evaluation of its median-size job with 1, 2, 4, 8 and 16 lanes per
// atom (CUDA events, reps evaluations each) and keep the fastest for every
// job of that dimension, present and future.
hdmd_status batch_autotune(hdmd_batch *b, int reps) {
    if (!b) return bfail(nullptr, HDMD_E_INVALID, "null batch");
    if (reps < 1) reps = 3;
    cudaStream_t s = b->stream;
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    for (int d = 2; d <= kMaxD; ++d) {
        std::vector<int> ids;
        for (int k = 0; k < b->max_jobs; ++k)
            if (b->jobs[k].live && b->jobs[k].d == d && b->h_jobs[k].status == JOB_ACTIVE) ids.push_back(k);
        if (ids.empty()) continue;
        std::sort(ids.begin(), ids.end(), [&](int a, int c) { return b->jobs[a].N < b->jobs[c].N; });
        const int id = ids[ids.size() / 2];
        BatchJob &J = b->h_jobs[id];
        float best = 1e30f;
        int best_lg = b->lgG[d];
        for (int lg = 0; lg <= 4; ++lg) {
            J.lgG = lg;
            J.built = 0;   // the list layout depends on the lanes per atom
            BCK(cudaMemcpyAsync(&b->d_jobs[id].lgG, &J.lgG, sizeof(int), cudaMemcpyHostToDevice, s));
            BCK(cudaMemcpyAsync(&b->d_jobs[id].built, &J.built, sizeof(int), cudaMemcpyHostToDevice, s));
            probe_one(d, b->d_jobs + id, 1, s);   // list build and warm-up
            BCK(cudaEventRecord(e0, s));
            probe_one(d, b->d_jobs + id, reps, s);
            BCK(cudaEventRecord(e1, s));
            BCK(cudaEventSynchronize(e1));
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; best_lg = lg; }
        }
        b->lgG[d] = best_lg;
        for (int k : ids) {
            // lists and forces are rebuilt in the chosen layout at the next run
            b->h_jobs[k].lgG = best_lg;
            b->h_jobs[k].built = 0;
            b->h_jobs[k].force_valid = 0;
            BCK(cudaMemcpyAsync(&b->d_jobs[k].built, &b->h_jobs[k].built, 3 * sizeof(int),
                                cudaMemcpyHostToDevice, s));
        }
        BCK(cudaStreamSynchronize(s));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return HDMD_OK;
}

hdmd_status batch_set_lanes(hdmd_batch *b, int d, int lanes) {
    if (!b) return bfail(nullptr, HDMD_E_INVALID, "null batch");
    if (d < 2 || d > kMaxD || lanes < 1 || lanes > 16 || (lanes & (lanes - 1)))
        return bfail(b, HDMD_E_INVALID, "lanes must be a power of two in 1..16");
    b->lgG[d] = __builtin_ctz(lanes);
    for (int k = 0; k < b->max_jobs; ++k) {
        if (!b->jobs[k].live || b->jobs[k].d != d) continue;
        b->h_jobs[k].lgG = b->lgG[d];
        b->h_jobs[k].built = 0;
        b->h_jobs[k].force_valid = 0;
        BCK(cudaMemcpyAsync(&b->d_jobs[k].built, &b->h_jobs[k].built, 3 * sizeof(int),
                            cudaMemcpyHostToDevice, b->stream));
    }
    BCK(cudaStreamSynchronize(b->stream));
    return HDMD_OK;
}

hdmd_status batch_destroy(hdmd_batch *b) {
    if (!b) return HDMD_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &kv : b->graphs) {
        cudaGraphExecDestroy(kv.second.second);
        cudaGraphDestroy(kv.second.first);
    }
    for (int k = 0; k < 2 * (kMaxD + 1); ++k) {
        if (b->fork[k]) cudaStreamDestroy(b->fork[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->pool_dev) cudaFree(b->pool_dev);
    if (b->d_jobs) cudaFree(b->d_jobs);
    if (b->d_order) cudaFree(b->d_order);
    if (b->d_ctl) cudaFree(b->d_ctl);
    if (b->h_jobs) cudaFreeHost(b->h_jobs);
    if (b->h_order) cudaFreeHost(b->h_order);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    cudaGetLastError();
    delete b;
    return HDMD_OK;
}

}  // extern "C"
