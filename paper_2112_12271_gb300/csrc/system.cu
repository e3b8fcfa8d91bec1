// system.cu -- host runtime and C ABI of the hdmd library (include/hdmd.h).
//
// Owns the device memory of a system, launches the kernels of the other
// translation units on the system's stream, and drives the loops of the
// method: the MD loop (Sec. II.B main loop with the Sec. II.C trigger) and
// the FIRE loop (Sec. II.B).  Both loops keep every decision on the device:
// the list rebuild is a CUDA-graph IF node whose condition the drift kernel
// sets, and the FIRE iteration is a WHILE node whose condition the force
// kernel sets after its FP64 reductions.  Without conditional-node support
// the same kernels run eagerly, the rebuild kernels returning at once
// unless the device-side trigger flag is set.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cstddef>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <utility>
#include <utility>
#include <vector>

#include "../../include/hdmd.h"
#include "launch.h"

using namespace hdmd;

namespace {

thread_local std::string g_thread_err;

struct GraphEx {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// Device memory of every system comes from one stream-ordered pool per
// device (cudaMallocFromPoolAsync / cudaFreeAsync on the system's stream).
// cudaFree and cudaFreeHost wait for the whole device, so with them one
// system's teardown would stall every system running on other streams;
// the pool keeps up to 4 GiB of freed memory for the next system.
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};

cudaMemPool_t device_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps pp = {};
        pp.allocType = cudaMemAllocationTypePinned;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = dev;
        cudaMemPool_t mp = nullptr;
        if (cudaMemPoolCreate(&mp, &pp) != cudaSuccess) return nullptr;
        uint64_t keep = 4ull << 30;
        cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = mp;
    }
    return g_pools[dev];
}

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t mp = device_pool();
    if (!mp) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes, mp, s);
}

void pool_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// Pinned host words for the flag and reduction read-backs: 1 KiB slots cut
// from 256 KiB pinned chunks that are kept for the life of the process, so
// that no system ever calls cudaFreeHost.
constexpr size_t kPinnedSlot = 1024;
std::mutex g_pinned_mu;
std::vector<char *> g_pinned_free;

void *pinned_get() {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    if (g_pinned_free.empty()) {
        char *chunk = nullptr;
        if (cudaMallocHost((void **)&chunk, 256 * kPinnedSlot) != cudaSuccess) return nullptr;
        for (int k = 255; k >= 0; --k) g_pinned_free.push_back(chunk + k * kPinnedSlot);
    }
    char *p = g_pinned_free.back();
    g_pinned_free.pop_back();
    return p;
}

void pinned_put(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    g_pinned_free.push_back((char *)p);
}

static_assert(sizeof(Flags) <= kPinnedSlot, "flag words exceed a pinned slot");
static_assert(sizeof(double) * kNRed <= kPinnedSlot, "reduction words exceed a pinned slot");

}  // namespace

struct hdmd_system {
    int d = 0;
    int64_t N = 0;
    double L = 0;
    hdmd_potential pot{};
    int prec = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr, cap_stream3 = nullptr;
    Dev dv{};
    std::vector<void *> allocs;
    int64_t bytes = 0;
    bool have_state = false;
    bool F_valid = false;
    bool rows32_valid = false, rows64_valid = false;
    int buf = 0;
    int use_graphs = 1;
    bool graphs_ok = true;
    std::string graph_err;
    double sigma_max = 0;
    double nvt_T = 0.0, nvt_tau = 0.0;   // Berendsen thermostat (tau <= 0: NVE)
    int rule = 0, n_bet = 1;             // list rebuild rule (0 exact, 1 the paper's)
    double baro_P = 0.0, baro_tau = 0.0, baro_beta = 0.0;   // Berendsen barostat
    int64_t baro_n = 0, baro_count = 0;
    int64_t cell_cap = 0;              // subcells the cell arrays hold
    double *obs_ref = nullptr;         // reference positions [N][d], caller order
    unsigned int *obs_hist = nullptr;  // G_s counts
    int obs_hist_cap = 0;
    bool unit_mass = true;
    double *inv_mass_store = nullptr;
    double *st_f = nullptr;
    // list storage (grown on overflow)
    int32_t *nbr = nullptr;
    uint32_t *code = nullptr;
    int64_t list_bytes = 0;
    // staging
    double *st_x = nullptr, *st_v = nullptr, *st_m = nullptr, *st_sig = nullptr;
    int32_t *st_i = nullptr, *st_cnt = nullptr, *st_idx = nullptr;
    int64_t st_idx_cap = 0;
    int64_t *st_off = nullptr;
    // snapshot for md_steps rollback
    double *snap_x0 = nullptr, *snap_dlt = nullptr, *snap_v = nullptr, *snap_sig = nullptr,
           *snap_im = nullptr;
    int32_t *snap_img = nullptr, *snap_id = nullptr;
    // pinned host mirror of flags and reductions
    Flags *h_flags = nullptr;
    double *h_red = nullptr;
    // graphs
    std::map<std::tuple<int, int, int, uint64_t>, GraphEx> md_graphs;  // (kind, len, in_buf, dt bits)
    std::map<int, GraphEx> fire_graphs;                                // fp64 phase -> graph
    // resident MD kernel (one cooperative launch per list; see kernels_resident.cu)
    int use_resident = 1;
    bool res_graph_ok = true;
    unsigned long long *res_sync = nullptr;   // [2][kResMaxGrid] step words, kResWordStride apart
    double *res_kin = nullptr;                // [2][kResMaxGrid] NVT partials
    // SWAP buffers (allocated on first use)
    SwapDev sw{};
    int sw_cap_pairs = 0;
    unsigned swap_round = 0;
    std::string err;
};

namespace {

hdmd_status fail(hdmd_system *s, hdmd_status code, const std::string &msg) {
    g_thread_err = msg;
    if (s) s->err = msg;
    return code;
}

#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return fail(sys, HDMD_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKL(sys)                                                                      \
    do {                                                                              \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess)                                                        \
            return fail(sys, HDMD_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
hdmd_status dalloc(hdmd_system *sys, T **p, size_t count) {
    size_t b = sizeof(T) * (count ? count : 1);
    void *q = nullptr;
    cudaError_t e = pool_alloc(&q, b, sys->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(sys, HDMD_E_NOMEM, std::string("device allocation of ") + std::to_string(b) +
                                           " bytes failed: " + cudaGetErrorString(e));
    }
    sys->allocs.push_back(q);
    sys->bytes += (int64_t)b;
    *p = (T *)q;
    return HDMD_OK;
}

#define DA(ptr, count)                                         \
    do {                                                       \
        hdmd_status st_ = dalloc(sys, &(ptr), (size_t)(count)); \
        if (st_ != HDMD_OK) return st_;                        \
    } while (0)

void free_graphs(hdmd_system *sys) {
    for (auto &kv : sys->md_graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    sys->md_graphs.clear();
    for (auto &kv : sys->fire_graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    sys->fire_graphs.clear();
}

int default_lanes(int64_t N) {
    if (N <= (1 << 17)) return 4;
    if (N <= (1 << 20)) return 2;
    return 1;
}

// expected longest list: atoms within max sigma + skin at the mean density,
// with head-room; the build reports the true maximum and the list grows.
int initial_capacity(int d, int64_t N, double L, double sigma_max, double skin) {
    const double rho = (double)N / std::pow(L, d);
    const double R = sigma_max + skin;
    const double vball = std::pow(M_PI, 0.5 * d) * std::pow(R, d) / std::tgamma(1.0 + 0.5 * d);
    double est = 1.6 * rho * vball + 16.0;
    est = std::min(est, (double)N + 8.0);
    return (int)est;
}

int initial_capacity(const hdmd_system *sys) {
    return initial_capacity(sys->d, sys->N, sys->L, sys->sigma_max, sys->pot.skin);
}

hdmd_status alloc_lists(hdmd_system *sys, int cap) {
    const int G = sys->dv.G;
    cap = ((cap + G - 1) / G) * G;
    if (cap < G) cap = G;
    if (sys->nbr) { pool_free(sys->nbr, sys->stream); sys->nbr = nullptr; }
    if (sys->code) { pool_free(sys->code, sys->stream); sys->code = nullptr; }
    sys->bytes -= sys->list_bytes;
    const size_t cnt = (size_t)cap * sys->dv.Npad;
    const bool packed = sys->dv.pack_sh > 0;   // one word per entry: no code array
    const size_t words = packed ? cnt : 2 * cnt;
    void *a = nullptr, *b = nullptr;
    cudaError_t e1 = pool_alloc(&a, cnt * sizeof(int32_t), sys->stream);
    cudaError_t e2 = (e1 == cudaSuccess && !packed) ? pool_alloc(&b, cnt * sizeof(uint32_t), sys->stream) : e1;
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        if (e1 == cudaSuccess) pool_free(a, sys->stream);
        sys->list_bytes = 0;
        return fail(sys, HDMD_E_NOMEM, "Verlet list allocation of " +
                                           std::to_string(words * 4) + " bytes failed");
    }
    sys->nbr = (int32_t *)a;
    sys->code = (uint32_t *)b;
    sys->list_bytes = (int64_t)(words * 4);
    sys->bytes += sys->list_bytes;
    sys->dv.nbr = sys->nbr;
    sys->dv.code = sys->code;
    sys->dv.cap = cap;
    free_graphs(sys);   // baked pointers changed
    return HDMD_OK;
}

hdmd_status read_flags(hdmd_system *sys) {
    CK(cudaMemcpyAsync(sys->h_flags, sys->dv.flags, sizeof(Flags), cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaMemcpyAsync(sys->h_red, sys->dv.red, sizeof(double) * kNRed, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    return HDMD_OK;
}

hdmd_status clear_flag_field(hdmd_system *sys, size_t offset, size_t bytes) {
    CK(cudaMemsetAsync((char *)sys->dv.flags + offset, 0, bytes, sys->stream));
    return HDMD_OK;
}

hdmd_status clear_errors(hdmd_system *sys) {
    hdmd_status st = clear_flag_field(sys, offsetof(Flags, error), sizeof(int) * 2);  // error, max_count
    if (st) return st;
    return clear_flag_field(sys, offsetof(Flags, rebuild), sizeof(int));
}

// unconditional list build; rows of buffer `buf` refreshed
hdmd_status rebuild_now(hdmd_system *sys, int buf) {
    launch_rebuild(sys->dv, buf, false, sys->stream);
    CKL(sys);
    sys->buf = buf;
    sys->rows32_valid = sys->rows64_valid = true;
    sys->F_valid = false;
    return HDMD_OK;
}

hdmd_status ensure_rows(hdmd_system *sys, int buf, bool need32, bool need64) {
    bool w32 = need32 && (!sys->rows32_valid || sys->buf != buf);
    bool w64 = need64 && (!sys->rows64_valid || sys->buf != buf);
    if (sys->buf != buf) {
        // the other kind is stale in the new buffer
        if (!need32) sys->rows32_valid = false;
        if (!need64) sys->rows64_valid = false;
    }
    if (w32 || w64) {
        launch_rows(sys->dv, buf, w32, w64, sys->stream);
        CKL(sys);
    }
    sys->buf = buf;
    if (need32) sys->rows32_valid = true;
    if (need64) sys->rows64_valid = true;
    return HDMD_OK;
}

hdmd_status check_device_errors(hdmd_system *sys) {
    if (sys->h_flags->error & ERR_LOST)
        return fail(sys, HDMD_E_LOST_ATOM,
                    "non-finite coordinates or a displacement beyond L/4 since the last list build");
    if (sys->h_flags->error & ERR_OVERFLOW)
        return fail(sys, HDMD_E_NBR_OVERFLOW, "Verlet list capacity exceeded");
    if (sys->h_flags->error & ERR_TIMEOUT)
        return fail(sys, HDMD_E_TIMEOUT, "a block of the resident MD kernel gave up waiting for the others");
    return HDMD_OK;
}

// grow the lists after an overflow seen by the last build(s)
hdmd_status grow_lists(hdmd_system *sys) {
    int need = sys->h_flags->max_count;
    int cap = (int)(need * 1.25) + 16;
    if (cap <= sys->dv.cap) cap = sys->dv.cap * 2;
    return alloc_lists(sys, cap);
}

hdmd_status build_forced(hdmd_system *sys, int buf) {
    for (int attempt = 0; attempt < 4; ++attempt) {
        hdmd_status st = clear_errors(sys);
        if (st) return st;
        st = rebuild_now(sys, buf);
        if (st) return st;
        st = read_flags(sys);
        if (st) return st;
        if (sys->h_flags->error & ERR_OVERFLOW) {
            st = grow_lists(sys);
            if (st) return st;
            continue;
        }
        return HDMD_OK;
    }
    return fail(sys, HDMD_E_NBR_OVERFLOW, "Verlet list kept overflowing after growing it");
}

// ----------------------------------------------------------------- graphs
// Conditional IF node on the capturing stream, body = a full list build.
hdmd_status add_if_rebuild(hdmd_system *sys, cudaStream_t cs, cudaGraphConditionalHandle h,
                           int buf, cudaStream_t body_stream) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
    CK(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeRelaxed));
    launch_rebuild(sys->dv, buf, false, body_stream);
    cudaGraph_t out = nullptr;
    CK(cudaStreamEndCapture(body_stream, &out));
    return HDMD_OK;
}

StepCfg base_cfg(const hdmd_system *sys, double dt) {
    StepCfg c;
    std::memset(&c, 0, sizeof(c));
    c.dt = dt;
    c.halfdt = 0.5 * dt;
    c.fp64_pairs = sys->prec == HDMD_FP64 ? 1 : 0;
    c.rule = sys->rule;
    c.n_bet = sys->n_bet;
    if (sys->nvt_tau > 0.0 && dt > 0.0) {
        c.nvt = 1;
        c.nvt_rate = dt / sys->nvt_tau;
        c.nvt_T = sys->nvt_T;
    }
    return c;
}

// kind 0: kick-drift from stored F, then IF rebuild (start of md_steps)
// kind 1: len x [force + kick + kick + drift, IF rebuild]
hdmd_status build_md_graph(hdmd_system *sys, int kind, int len, int in_buf, double dt,
                           GraphEx *out) {
    cudaStream_t cs = sys->cap_stream;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr);
    hdmd_status st = HDMD_OK;
    int cur = in_buf;
    const int steps = kind == 0 ? 1 : len;
    for (int k = 0; k < steps && e == cudaSuccess && st == HDMD_OK; ++k) {
        cudaGraphConditionalHandle h;
        e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) break;
        StepCfg c = base_cfg(sys, dt);
        c.compute_force = kind == 0 ? 0 : 1;
        c.kick2 = kind == 0 ? 0 : 1;
        c.kick1_drift = 1;
        c.in_buf = cur;
        c.out_buf = 1 - cur;
        c.cond_rebuild = h;
        launch_step(sys->dv, c, cs);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        st = add_if_rebuild(sys, cs, h, 1 - cur, sys->cap_stream2);
        cur = 1 - cur;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (st != HDMD_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(sys, HDMD_E_CUDA, std::string("graph capture: ") +
                                          cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(sys, HDMD_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    out->graph = graph;
    out->exec = ex;
    return HDMD_OK;
}

uint64_t dbits(double x) { uint64_t b; std::memcpy(&b, &x, 8); return b; }

hdmd_status run_md_piece(hdmd_system *sys, int kind, int len, int in_buf, double dt) {
    if (sys->use_graphs && sys->graphs_ok) {
        auto key = std::make_tuple(kind, len, in_buf, dbits(dt));
        auto it = sys->md_graphs.find(key);
        if (it == sys->md_graphs.end()) {
            GraphEx ge;
            hdmd_status st = build_md_graph(sys, kind, len, in_buf, dt, &ge);
            if (st != HDMD_OK) {
                sys->graphs_ok = false;   // fall back to eager launches from now on
                sys->graph_err = sys->err;
                g_thread_err.clear();
                sys->err.clear();
            } else {
                it = sys->md_graphs.emplace(key, ge).first;
            }
        }
        if (sys->graphs_ok) {
            CK(cudaGraphLaunch(it->second.exec, sys->stream));
            return HDMD_OK;
        }
    }
    // eager: the rebuild kernels check the device-side trigger themselves
    int cur = in_buf;
    const int steps = kind == 0 ? 1 : len;
    for (int k = 0; k < steps; ++k) {
        StepCfg c = base_cfg(sys, dt);
        c.compute_force = kind == 0 ? 0 : 1;
        c.kick2 = kind == 0 ? 0 : 1;
        c.kick1_drift = 1;
        c.in_buf = cur;
        c.out_buf = 1 - cur;
        launch_step(sys->dv, c, sys->stream);
        launch_rebuild(sys->dv, 1 - cur, true, sys->stream);
        CKL(sys);
        cur = 1 - cur;
    }
    return HDMD_OK;
}

hdmd_status force_only(hdmd_system *sys, int buf, bool fp64, bool thermo) {
    StepCfg c = base_cfg(sys, 0.0);
    c.fp64_pairs = fp64 ? 1 : 0;
    c.compute_force = 1;
    c.store_F = 1;
    c.thermo = thermo ? 1 : 0;
    c.in_buf = buf;
    c.out_buf = buf;
    launch_step(sys->dv, c, sys->stream);
    CKL(sys);
    return HDMD_OK;
}

void fill_thermo(const hdmd_system *sys, const double *red, hdmd_thermo *t) {
    const double K = 0.5 * red[R_K2];
    const double W = 0.5 * red[R_W];
    t->E_pair = 0.5 * red[R_E];
    t->virial = W;
    t->K = K;
    t->T = 2.0 * K / (sys->d * (double)(sys->N - 1));
    t->P = (2.0 * K + W) / (sys->d * std::pow(sys->L, sys->d));
}

hdmd_status snapshot(hdmd_system *sys, bool restore) {
    const size_t nd = (size_t)sys->d * sys->dv.Npad, n = sys->dv.Npad;
    auto cp = [&](void *dst, const void *src, size_t b) {
        return cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToDevice, sys->stream);
    };
    Dev &dv = sys->dv;
    if (!restore) {
        CK(cp(sys->snap_x0, dv.x0, nd * 8));
        CK(cp(sys->snap_dlt, dv.dlt, nd * 8));
        CK(cp(sys->snap_v, dv.v, nd * 8));
        CK(cp(sys->snap_img, dv.img, nd * 4));
        CK(cp(sys->snap_id, dv.id, n * 4));
        CK(cp(sys->snap_sig, dv.sigma, n * 8));
        if (dv.inv_mass) CK(cp(sys->snap_im, dv.inv_mass, n * 8));
    } else {
        CK(cp(dv.x0, sys->snap_x0, nd * 8));
        CK(cp(dv.dlt, sys->snap_dlt, nd * 8));
        CK(cp(dv.v, sys->snap_v, nd * 8));
        CK(cp(dv.img, sys->snap_img, nd * 4));
        CK(cp(dv.id, sys->snap_id, n * 4));
        CK(cp(dv.sigma, sys->snap_sig, n * 8));
        if (dv.inv_mass) CK(cp(dv.inv_mass, sys->snap_im, n * 8));
    }
    return HDMD_OK;
}

// Berendsen factor of the first step of an md_steps call, from the kinetic
// temperature of the current velocities (a force pass with the thermo sums)
hdmd_status nvt_prepare(hdmd_system *sys, int buf, bool fp64, double dt) {
    hdmd_status st = force_only(sys, buf, fp64, true);
    if (st) return st;
    st = read_flags(sys);
    if (st) return st;
    const double T = sys->h_red[R_K2] / ((double)sys->d * (double)(sys->N - 1));
    const double rate = dt / sys->nvt_tau;
    sys->h_flags->nvt_lambda = T > 0.0 ? std::sqrt(std::max(0.0, 1.0 + rate * (sys->nvt_T / T - 1.0))) : 1.0;
    sys->h_flags->nvt_T = T;
    CK(cudaMemcpyAsync(&sys->dv.flags->nvt_lambda, &sys->h_flags->nvt_lambda, 2 * sizeof(double),
                       cudaMemcpyHostToDevice, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    return HDMD_OK;
}

constexpr int kChunk = 64;

// ----------------------------------------------------------------- resident MD
// Launch shape of the resident kernel for the current system: grid (at most
// one block per SM, at least 64 atoms per block), atoms per block and the
// shared memory, whose remainder after the per-atom arrays holds the lists.
// False where the path does not apply (FP64 pairs, the paper's rebuild rule,
// no cooperative launch, or per-atom arrays too large for shared memory):
// md_steps then launches one kernel per step.
struct ResPlan {
    int grid = 0, na_cap = 0, list_cap = 0;
    size_t smem = 0;
};

bool resident_plan(hdmd_system *sys, ResPlan *p) {
    if (!sys->use_resident || sys->prec != HDMD_MIXED || sys->rule != 0) return false;
    int dev = 0, sms = 0, optin = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (!coop) return false;
    const int64_t N = sys->N;
    int grid = (int)std::min<int64_t>(std::min(sms, kResMaxGrid), std::max<int64_t>(1, N / 64));
    const int na_cap = (int)((N + grid - 1) / grid);
    const bool pack = sys->d <= kMaxPackD && sys->dv.pack_sh > 0;
    const size_t word = pack ? 4 : 8;
    const size_t fixed = resident_fixed_smem(sys->d, na_cap, pack);
    const size_t static_smem = 10 * 1024;   // the kernel's own shared arrays
    if ((size_t)optin < static_smem + fixed + 16 * word * (size_t)na_cap) return false;
    const size_t budget = (size_t)optin - static_smem;
    const size_t list_cap = std::min((budget - fixed) / word, (size_t)na_cap * (size_t)sys->dv.cap);
    const size_t smem = (fixed + list_cap * word + 15) & ~(size_t)15;
    int occ = 0;
    if (resident_occupancy(sys->dv, smem, &occ) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return false;
    }
    p->grid = grid;
    p->na_cap = na_cap;
    p->list_cap = (int)list_cap;
    p->smem = smem;
    return true;
}

ResCfg resident_cfg(const hdmd_system *sys, const ResPlan &p, int in_buf, double dt) {
    ResCfg rc;
    std::memset(&rc, 0, sizeof(rc));
    rc.dt = dt;
    rc.halfdt = 0.5 * dt;
    rc.in_buf = in_buf;
    if (sys->nvt_tau > 0.0) {
        rc.nvt = 1;
        rc.nvt_rate = dt / sys->nvt_tau;
        rc.nvt_T = sys->nvt_T;
    }
    rc.na_cap = p.na_cap;
    rc.list_cap = p.list_cap;
    rc.spin_limit = 1 << 21;   // ~0.1-1 s of polling: ERR_TIMEOUT after it
    rc.sync = sys->res_sync;
    rc.kin = sys->res_kin;
    return rc;
}

// WHILE(steps left) { resident kernel; IF(trigger) list build }
hdmd_status build_res_graph(hdmd_system *sys, const ResPlan &pl, int in_buf, double dt,
                            GraphEx *out) {
    cudaStream_t cs = sys->cap_stream, cs2 = sys->cap_stream2;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    hdmd_status st = HDMD_OK;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr);
    cudaGraphConditionalHandle hw = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault);
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &nd);
    cudaGraphNode_t node;
    cudaGraphNodeParams p = {};
    if (e == cudaSuccess) {
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = hw;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p);
    }
    if (e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
        cudaGraph_t body = p.conditional.phGraph_out[0];
        cudaGraphConditionalHandle hi = 0;
        e = cudaGraphConditionalHandleCreate(&hi, body, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            ResCfg rc = resident_cfg(sys, pl, in_buf, dt);
            rc.cond_loop = hw;
            rc.cond_rebuild = hi;
            e = launch_md_resident(sys->dv, rc, pl.grid, pl.smem, cs2);
            if (e == cudaSuccess) st = add_if_rebuild(sys, cs2, hi, in_buf, sys->cap_stream3);
            cudaGraph_t bo = nullptr;
            cudaError_t e3 = cudaStreamEndCapture(cs2, &bo);
            if (e == cudaSuccess) e = e3;
        }
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (st != HDMD_OK || e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (st != HDMD_OK) return st;
        return fail(sys, HDMD_E_CUDA, std::string("resident graph capture: ") +
                                          cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(sys, HDMD_E_CUDA, std::string("resident graph instantiate: ") + cudaGetErrorString(e));
    }
    out->graph = graph;
    out->exec = ex;
    return HDMD_OK;
}

// nsteps middle MD steps (force, both kicks, drift) through the resident
// kernel, rows in and out of gather buffer in_buf; lists rebuilt whenever the
// trigger fires
hdmd_status run_resident(hdmd_system *sys, const ResPlan &pl, int64_t nsteps, int in_buf, double dt) {
    launch_set_res_left(sys->dv, nsteps, sys->stream);
    CKL(sys);
    if (sys->use_graphs && sys->graphs_ok && sys->res_graph_ok) {
        auto key = std::make_tuple(2, 0, in_buf, dbits(dt));
        auto it = sys->md_graphs.find(key);
        if (it == sys->md_graphs.end()) {
            GraphEx ge;
            hdmd_status st = build_res_graph(sys, pl, in_buf, dt, &ge);
            if (st != HDMD_OK) {
                sys->res_graph_ok = false;   // the eager loop below from now on
                sys->graph_err = sys->err;
                g_thread_err.clear();
                sys->err.clear();
            } else {
                it = sys->md_graphs.emplace(key, ge).first;
            }
        }
        if (sys->res_graph_ok) {
            CK(cudaGraphLaunch(it->second.exec, sys->stream));
            return HDMD_OK;
        }
    }
    const ResCfg rc = resident_cfg(sys, pl, in_buf, dt);
    for (;;) {
        CK(launch_md_resident(sys->dv, rc, pl.grid, pl.smem, sys->stream));
        launch_rebuild(sys->dv, in_buf, true, sys->stream);
        CKL(sys);
        hdmd_status st = read_flags(sys);
        if (st) return st;
        if (sys->h_flags->res_left <= 0 || sys->h_flags->error) return HDMD_OK;
    }
}

hdmd_status md_once(hdmd_system *sys, int64_t nsteps, double dt, hdmd_thermo *last) {
    hdmd_status st = clear_errors(sys);
    if (st) return st;
    int nb0;
    CK(cudaMemcpyAsync(&sys->h_flags->nbuilds, &sys->dv.flags->nbuilds, sizeof(int),
                       cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    nb0 = sys->h_flags->nbuilds;
    const bool fp64 = sys->prec == HDMD_FP64;
    st = ensure_rows(sys, sys->buf, !fp64, fp64);
    if (st) return st;
    if (!sys->F_valid) {
        st = force_only(sys, sys->buf, fp64, false);
        if (st) return st;
        sys->F_valid = true;
    }
    if (sys->nvt_tau > 0.0 && nsteps > 0) {
        st = nvt_prepare(sys, sys->buf, fp64, dt);
        if (st) return st;
    }
    int cur = sys->buf;
    ResPlan pl;
    if (nsteps > 0) {
        st = run_md_piece(sys, 0, 1, cur, dt);
        if (st) return st;
        cur = 1 - cur;
        int64_t left = nsteps - 1;
        if (left > 0 && resident_plan(sys, &pl)) {
            st = run_resident(sys, pl, left, cur, dt);
            if (st) return st;
            left = 0;
        }
        while (left > 0) {
            int len = (int)std::min<int64_t>(left, kChunk);
            st = run_md_piece(sys, 1, len, cur, dt);
            if (st) return st;
            if (len & 1) cur = 1 - cur;
            left -= len;
        }
    }
    // final force, second half kick, thermo
    StepCfg c = base_cfg(sys, dt);
    c.compute_force = 1;
    c.kick2 = nsteps > 0 ? 1 : 0;
    c.store_F = 1;
    c.thermo = 1;
    c.in_buf = cur;
    c.out_buf = cur;
    launch_step(sys->dv, c, sys->stream);
    CKL(sys);
    sys->buf = cur;
    if (fp64) { sys->rows64_valid = true; sys->rows32_valid = false; }
    else { sys->rows32_valid = true; sys->rows64_valid = false; }
    sys->F_valid = true;
    st = read_flags(sys);
    if (st) return st;
    if (last) {
        fill_thermo(sys, sys->h_red, last);
        last->steps = nsteps;
        last->rebuilds = sys->h_flags->nbuilds - nb0;
    }
    return check_device_errors(sys);
}


// ----------------------------------------------------------------- FIRE
StepCfg fire_force_cfg(const hdmd_system *sys, bool fp64, unsigned long long cond_loop) {
    StepCfg c = base_cfg(sys, 0.0);
    c.fp64_pairs = fp64 ? 1 : 0;
    c.compute_force = 1;
    c.store_F = 1;
    c.fire_red = 1;
    c.in_buf = 0;
    c.out_buf = 0;
    c.cond_loop = cond_loop;
    return c;
}

// [force + FIRE scalars] then WHILE(running) { update; IF(trigger) build; force + scalars }
hdmd_status build_fire_graph(hdmd_system *sys, bool fp64, GraphEx *out) {
    cudaStream_t cs = sys->cap_stream, cs2 = sys->cap_stream2;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    hdmd_status st = HDMD_OK;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr);
    cudaGraphConditionalHandle hw = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hw, g, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        launch_step(sys->dv, fire_force_cfg(sys, fp64, hw), cs);
        e = cudaGetLastError();
    }
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &nd);
    cudaGraphNode_t node;
    cudaGraphNodeParams p = {};
    if (e == cudaSuccess) {
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = hw;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p);
    }
    if (e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
        cudaGraph_t body = p.conditional.phGraph_out[0];
        cudaGraphConditionalHandle hi = 0;
        e = cudaGraphConditionalHandleCreate(&hi, body, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            launch_fire_update(sys->dv, fp64 ? 1 : 0, hi, cs2);
            e = cudaGetLastError();
            if (e == cudaSuccess) st = add_if_rebuild(sys, cs2, hi, 0, sys->cap_stream3);
            if (e == cudaSuccess && st == HDMD_OK) {
                launch_step(sys->dv, fire_force_cfg(sys, fp64, hw), cs2);
                e = cudaGetLastError();
            }
            cudaGraph_t bo = nullptr;
            cudaError_t e3 = cudaStreamEndCapture(cs2, &bo);
            if (e == cudaSuccess) e = e3;
        }
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (st != HDMD_OK || e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (st != HDMD_OK) return st;
        return fail(sys, HDMD_E_CUDA, std::string("FIRE graph capture: ") +
                                          cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(sys, HDMD_E_CUDA, std::string("FIRE graph instantiate: ") + cudaGetErrorString(e));
    }
    out->graph = graph;
    out->exec = ex;
    return HDMD_OK;
}

hdmd_status read_fire(hdmd_system *sys) {
    CK(cudaMemcpyAsync(sys->h_flags, sys->dv.flags, sizeof(Flags), cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    return HDMD_OK;
}

// one FIRE phase with FP32 or FP64 pair forces, until the status leaves RUNNING
hdmd_status fire_phase(hdmd_system *sys, bool fp64) {
    if (sys->use_graphs && sys->graphs_ok) {
        auto it = sys->fire_graphs.find(fp64 ? 1 : 0);
        if (it == sys->fire_graphs.end()) {
            GraphEx ge;
            hdmd_status st = build_fire_graph(sys, fp64, &ge);
            if (st != HDMD_OK) {
                sys->graphs_ok = false;
                sys->graph_err = sys->err;
                g_thread_err.clear();
                sys->err.clear();
            } else {
                it = sys->fire_graphs.emplace(fp64 ? 1 : 0, ge).first;
            }
        }
        if (sys->graphs_ok) {
            CK(cudaGraphLaunch(it->second.exec, sys->stream));
            return read_fire(sys);
        }
    }
    // eager: fixed bursts of iterations, every kernel returning at once after the end
    launch_step(sys->dv, fire_force_cfg(sys, fp64, 0), sys->stream);
    CKL(sys);
    for (;;) {
        for (int k = 0; k < 32; ++k) {
            launch_fire_update(sys->dv, fp64 ? 1 : 0, 0, sys->stream);
            launch_rebuild(sys->dv, 0, true, sys->stream);
            launch_step(sys->dv, fire_force_cfg(sys, fp64, 0), sys->stream);
        }
        CKL(sys);
        hdmd_status st = read_fire(sys);
        if (st) return st;
        if (sys->h_flags->fire[FS_STATUS] != (double)FIRE_RUNNING) return HDMD_OK;
    }
}

hdmd_status fire_once(hdmd_system *sys, const hdmd_fire_params &p, hdmd_fire_result *res) {
    Dev &dv = sys->dv;
    hdmd_status st = clear_errors(sys);
    if (st) return st;
    CK(cudaMemsetAsync(dv.v, 0, sizeof(double) * sys->d * dv.Npad, sys->stream));
    const bool mixed = sys->prec == HDMD_MIXED;
    double fs[FS_COUNT] = {0};
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
    // FP32 pair forces resolve max|F| down to about (pair stiffness) x (FP32
    // position resolution): the switch threshold scales with the law's
    // stiffness at contact relative to the harmonic law's, 1 (harmonic),
    // 2 (a sigma_max)^2 (Morse, Eq. (1)) or 2 n^2 (Mie)
    const double stiff = sys->dv.law == 1 ? 2.0 * (sys->dv.morse_a * sys->sigma_max) *
                                                (sys->dv.morse_a * sys->sigma_max)
                       : sys->dv.law == 2 ? 2.0 * sys->dv.mie_n * sys->dv.mie_n
                                          : 1.0;
    fs[FP_SWITCH] = (mixed && p.polish_tol > p.f_tol) ? p.polish_tol * stiff : 0.0;
    fs[FP_NDELAY] = (double)p.n_delay;
    fs[FP_NNEGMAX] = (double)p.n_neg_max;
    fs[FP_MAXITER] = (double)p.max_iter;
    fs[FP_INITDELAY] = p.initial_delay ? 1.0 : 0.0;
    fs[FP_ETHRES] = p.e_thres;
    fs[FP_FTHRES] = p.f_thres;
    fs[FP_DXMAX] = p.dx_max;
    fs[FP_NATOMS] = (double)sys->N;
    fs[FS_FITER] = -1.0;
    std::memcpy(sys->h_flags->fire, fs, sizeof(fs));
    CK(cudaMemcpyAsync(dv.flags->fire, sys->h_flags->fire, sizeof(fs), cudaMemcpyHostToDevice, sys->stream));
    CK(cudaMemcpyAsync(&sys->h_flags->nbuilds, &dv.flags->nbuilds, sizeof(int), cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    const int nb0 = sys->h_flags->nbuilds;
    bool fp64 = !mixed;
    st = ensure_rows(sys, 0, true, fp64);
    if (st) return st;
    st = fire_phase(sys, fp64);
    if (st) return st;
    int64_t polish = 0;
    if (sys->h_flags->fire[FS_STATUS] == (double)FIRE_SWITCH && !(sys->h_flags->error & (ERR_LOST | ERR_OVERFLOW))) {
        // continue the same FIRE iteration with FP64 pair forces
        sys->h_flags->fire[FP_SWITCH] = 0.0;
        sys->h_flags->fire[FS_STATUS] = FIRE_RUNNING;
        sys->h_flags->fire[FS_PHASE_ITER] = 0.0;
        sys->h_flags->fire[FS_NNEG] = 0.0;
        sys->h_flags->fire[FS_NPOS] = 0.0;
        CK(cudaMemcpyAsync(dv.flags->fire, sys->h_flags->fire, sizeof(double) * FS_COUNT,
                           cudaMemcpyHostToDevice, sys->stream));
        sys->rows64_valid = false;
        st = ensure_rows(sys, 0, true, true);
        if (st) return st;
        fp64 = true;
        st = fire_phase(sys, true);
        if (st) return st;
        polish = (int64_t)sys->h_flags->fire[FS_PHASE_ITER];
    }
    sys->buf = 0;
    sys->rows32_valid = true;
    sys->rows64_valid = fp64;
    sys->F_valid = true;
    const double *f = sys->h_flags->fire;
    if (res) {
        res->iterations = (int64_t)f[FS_ITER];
        res->polish_iterations = polish;
        res->rebuilds = sys->h_flags->nbuilds - nb0;
        res->E_pair = f[FS_E];
        res->fmax = f[FS_FMAX];
        res->converged = f[FS_STATUS] == (double)FIRE_CONVERGED;
    }
    st = check_device_errors(sys);
    if (st) return st;
    if (f[FS_STATUS] != (double)FIRE_CONVERGED) {
        const int s = (int)f[FS_STATUS];
        return fail(sys, HDMD_E_NOT_CONVERGED,
                    s == FIRE_MAXITER ? "FIRE reached max_iter" : "FIRE stopped: too many P <= 0 steps or non-finite forces");
    }
    return HDMD_OK;
}


// ----------------------------------------------------------------- SWAP
hdmd_status swap_alloc(hdmd_system *sys, int npairs, int scap) {
    SwapDev &sw = sys->sw;
    if (npairs <= sys->sw_cap_pairs && scap <= sw.scap) return HDMD_OK;
    cudaStream_t s = sys->stream;
    auto rel = [s](void *p) { pool_free(p, s); };
    auto get = [s](auto **p, size_t bytes) {
        void *q = nullptr;
        const bool ok = pool_alloc(&q, bytes, s) == cudaSuccess;
        *p = ok ? reinterpret_cast<typename std::remove_reference<decltype(**p)>::type *>(q) : nullptr;
        return ok;
    };
    if (npairs > sys->sw_cap_pairs) {
        rel(sw.ids); rel(sw.u); rel(sw.pairs); rel(sw.state); rel(sw.scount);
        sw.ids = nullptr; sw.u = nullptr; sw.pairs = nullptr; sw.state = nullptr; sw.scount = nullptr;
        if (!get(&sw.ids, sizeof(int32_t) * 2 * npairs) ||
            !get(&sw.u, sizeof(double) * npairs) ||
            !get(&sw.pairs, sizeof(int32_t) * 2 * npairs) ||
            !get(&sw.state, npairs) ||
            !get(&sw.scount, sizeof(int32_t) * 2 * npairs)) {
            cudaGetLastError();
            sys->sw_cap_pairs = 0;
            return fail(sys, HDMD_E_NOMEM, "SWAP pair buffers");
        }
        sys->sw_cap_pairs = npairs;
        rel(sw.slist);
        sw.slist = nullptr;
        sw.scap = 0;
    }
    if (!sw.owner) {
        if (!get(&sw.owner, sizeof(unsigned long long) * sys->dv.Npad) ||
            !get(&sw.slot_of, sizeof(int32_t) * sys->dv.Npad) ||
            !get(&sw.overflow, sizeof(int) * 4) ||
            !get(&sw.nacc, sizeof(unsigned long long))) {
            cudaGetLastError();
            return fail(sys, HDMD_E_NOMEM, "SWAP owner buffers");
        }
        sw.npend = sw.overflow + 1;
        CK(cudaMemsetAsync(sw.owner, 0xFF, sizeof(unsigned long long) * sys->dv.Npad, sys->stream));
    }
    if (scap > sw.scap || !sw.slist) {
        rel(sw.slist);
        sw.slist = nullptr;
        if (!get(&sw.slist, sizeof(int32_t) * (size_t)2 * sys->sw_cap_pairs * scap)) {
            cudaGetLastError();
            sw.scap = 0;
            return fail(sys, HDMD_E_NOMEM, "SWAP neighbour lists");
        }
        sw.scap = scap;
    }
    return HDMD_OK;
}

void swap_free(hdmd_system *sys) {
    SwapDev &sw = sys->sw;
    for (void *p : {(void *)sw.ids, (void *)sw.u, (void *)sw.pairs, (void *)sw.state, (void *)sw.owner,
                    (void *)sw.slot_of, (void *)sw.slist, (void *)sw.scount, (void *)sw.overflow,
                    (void *)sw.nacc})
        pool_free(p, sys->stream);
    sw = SwapDev{};
}

int swap_list_estimate(const hdmd_system *sys) {
    const int d = sys->d;
    const double rho = (double)sys->N / std::pow(sys->L, d);
    const double R = sys->sigma_max;
    const double vball = std::pow(M_PI, 0.5 * d) * std::pow(R, d) / std::tgamma(1.0 + 0.5 * d);
    return (int)std::min(2.0 * rho * vball + 32.0, (double)sys->N + 1.0);
}

// one pass over the candidates already in sw.ids / sw.u
hdmd_status swap_pass(hdmd_system *sys) {
    SwapDev &sw = sys->sw;
    for (int attempt = 0; attempt < 6; ++attempt) {
        CK(cudaMemsetAsync(sw.overflow, 0, sizeof(int), sys->stream));
        launch_swap_prepare(sys->dv, sw, sys->buf, sys->stream);
        CKL(sys);
        int ov = 0;
        CK(cudaMemcpyAsync(&sys->h_flags->pad0, sw.overflow, sizeof(int), cudaMemcpyDeviceToHost, sys->stream));
        CK(cudaStreamSynchronize(sys->stream));
        ov = sys->h_flags->pad0;
        if (ov == 0) break;
        hdmd_status st = swap_alloc(sys, sys->sw_cap_pairs, (int)(ov * 1.25) + 16);
        if (st) return st;
        if (attempt == 5) return fail(sys, HDMD_E_NBR_OVERFLOW, "SWAP neighbour lists kept overflowing");
    }
    const int64_t max_rounds = (int64_t)sw.npairs + 2;
    int64_t done_rounds = 0;
    for (;;) {
        const int burst = 8;
        for (int r = 0; r < burst; ++r) {
            if (r == burst - 1) CK(cudaMemsetAsync(sw.npend, 0, sizeof(int), sys->stream));
            launch_swap_round(sys->dv, sw, sys->swap_round++, sys->stream);
        }
        CKL(sys);
        done_rounds += burst;
        CK(cudaMemcpyAsync(&sys->h_flags->pad0, sw.npend, sizeof(int), cudaMemcpyDeviceToHost, sys->stream));
        CK(cudaStreamSynchronize(sys->stream));
        if (sys->h_flags->pad0 == 0) return HDMD_OK;
        if (done_rounds > max_rounds + burst)
            return fail(sys, HDMD_E_TIMEOUT, "SWAP rounds did not finish");
    }
}

hdmd_status validate_sys(hdmd_system *sys) {
    if (!sys) return fail(nullptr, HDMD_E_INVALID, "null system");
    if (!sys->have_state) return fail(sys, HDMD_E_INVALID, "set_state must be called first");
    return HDMD_OK;
}

// Argument checks of create_system; on success the largest diameter and the
// subcells per axis.
hdmd_status check_create_args(int d, int64_t N, double L, const double *diameters,
                              const hdmd_potential *pot, hdmd_precision prec, double *smax_out,
                              int *n_out) {
    if (d < 2 || d > kMaxD) return fail(nullptr, HDMD_E_UNSUPPORTED_D, "d must be in 2..10");
    if (N < 2 || N > (int64_t)1 << 28) return fail(nullptr, HDMD_E_INVALID, "N must be in 2..2^28");
    if (!(L > 0.0) || !std::isfinite(L)) return fail(nullptr, HDMD_E_INVALID, "L must be positive and finite");
    if (!diameters) return fail(nullptr, HDMD_E_INVALID, "diameters is NULL");
    if (!pot) return fail(nullptr, HDMD_E_INVALID, "potential is NULL");
    if (pot->kind < 0 || pot->kind > 2)
        return fail(nullptr, HDMD_E_INVALID, "pair law kind must be 0 (harmonic), 1 (Morse) or 2 (Mie)");
    if (pot->kind == 2 && (pot->n_mie < 1 || pot->n_mie > 24))
        return fail(nullptr, HDMD_E_INVALID, "the Mie exponent n_mie must be in 1..24");
    if (pot->kind == 1 && (!(pot->a > 0.0) || !std::isfinite(pot->a)))
        return fail(nullptr, HDMD_E_INVALID, "the Morse stiffness a must be positive and finite");
    if (pot->eps_scale != 0 && pot->eps_scale != 1)
        return fail(nullptr, HDMD_E_INVALID, "eps_scale must be 0 or 1");
    if (!(pot->eps > 0.0) || !std::isfinite(pot->eps)) return fail(nullptr, HDMD_E_INVALID, "eps must be positive");
    if (!(pot->skin >= 0.0) || !std::isfinite(pot->skin)) return fail(nullptr, HDMD_E_INVALID, "skin must be >= 0");
    if (prec != HDMD_FP64 && prec != HDMD_MIXED) return fail(nullptr, HDMD_E_INVALID, "unknown precision");
    double smax = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        if (!(diameters[i] > 0.0) || !std::isfinite(diameters[i]))
            return fail(nullptr, HDMD_E_INVALID, "diameters must be positive and finite");
        smax = std::max(smax, diameters[i]);
    }
    const double rc = smax + pot->skin;
    // only one periodic image of a pair may interact: L > 2 max diameter
    if (!(L > 2.0 * smax))
        return fail(nullptr, HDMD_E_INVALID, "box too small: L must exceed twice the largest diameter");
    int n = std::max(1, (int)std::floor(L / rc));   // Eq. (7); 1: a single subcell, all pairs
    // larger subcells stay exact; cap the subcell count at ~8N (+4096)
    const double cap_cells = 8.0 * (double)N + 4096.0;
    while (n > 2 && std::pow((double)n, d) > cap_cells) --n;
    if (std::pow((double)n, d) > 2.0e9) return fail(nullptr, HDMD_E_INVALID, "too many subcells");

    *smax_out = smax;
    *n_out = n;
    return HDMD_OK;
}

// Index bits of a list entry when the stencil position fits beside them in
// one 32-bit word (packed entries), else 0.
int pack_shift(int d, int64_t Npad) {
    int sh = 1;
    while (((int64_t)1 << sh) < Npad) ++sh;
    return (HDMD_PACK_LISTS && d <= kMaxPackD && stencil_bits(d) + sh <= 32) ? sh : 0;
}

// Bytes of the arrays create_system allocates, in its order and with the
// same rounding as dalloc, plus the list arrays at capacity cap (one word per
// entry when packed, two otherwise).
int64_t create_bytes(int d, int64_t N, int64_t ncells, int cap, int G) {
    const size_t Np = (size_t)((N + 63) / 64 * 64), nd = (size_t)d * Np;
    const size_t RF = kRowFloats(d), RD = kRowDoubles(d);
    const size_t maxblocks = (Np * kMaxLanes + kStepNT - 1) / kStepNT;
    const size_t nc = (size_t)ncells;
    int64_t b = 0;
    auto fb = [&b](size_t elem, size_t count) { b += (int64_t)(elem * (count ? count : 1)); };
#define FB(m, count) fb(sizeof(*std::declval<Dev &>().m), (size_t)(count))
#define SB(m, count) fb(sizeof(*std::declval<hdmd_system &>().m), (size_t)(count))
    FB(x0, nd); FB(dlt, nd); FB(v, nd); FB(F, nd);
    FB(sigma, Np); SB(inv_mass_store, Np); SB(st_f, nd);
    FB(img, nd); FB(id, Np);
    FB(gs0, Np * RF); FB(gs[0], Np * RF); FB(gs[1], Np * RF);
    FB(gd[0], Np * RD); FB(gd[1], Np * RD);
    FB(cell_count, nc); FB(cell_fill, nc); FB(cell_start, nc + 1);
    FB(cell_of, Np); FB(perm, Np); FB(cellid, Np); FB(batch_start, nc + 1);
    FB(tx, nd); FB(tv, nd); FB(tsig, Np); FB(tim, Np);
    FB(timg, nd); FB(tid, Np);
    FB(nnbr, Np);
    FB(partials, (size_t)kNRed * maxblocks);
    FB(red, kNRed);
    FB(flags, 1);
    SB(st_x, nd); SB(st_v, nd); SB(st_m, Np); SB(st_sig, Np);
    SB(st_i, nd); SB(st_cnt, Np); SB(st_off, Np + 1);
    SB(snap_x0, nd); SB(snap_dlt, nd); SB(snap_v, nd); SB(snap_sig, Np);
    SB(snap_im, Np); SB(snap_img, nd); SB(snap_id, Np);
    SB(res_sync, 2 * kResMaxGrid * kResWordStride); SB(res_kin, 2 * kResMaxGrid);
#undef FB
#undef SB
    int64_t c = ((int64_t)(cap + G - 1) / G) * G;
    if (c < G) c = G;
    const int64_t words = pack_shift(d, (int64_t)Np) ? 1 : 2;   // nbr (and code)
    b += (int64_t)sizeof(int32_t) * words * c * (int64_t)Np;
    return b;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

hdmd_status system_footprint(int d, int64_t N, double L, const double *diameters,
                             const hdmd_potential *pot, hdmd_precision prec, int64_t *bytes) {
    if (!bytes) return fail(nullptr, HDMD_E_INVALID, "bytes is NULL");
    double smax = 0.0;
    int n = 1;
    hdmd_status st = check_create_args(d, N, L, diameters, pot, prec, &smax, &n);
    if (st) return st;
    int64_t ncells = 1;
    for (int k = 0; k < d; ++k) ncells *= n;
    *bytes = create_bytes(d, N, ncells, initial_capacity(d, N, L, smax, pot->skin), default_lanes(N));
    return HDMD_OK;
}

hdmd_status create_system(int d, int64_t N, double L, const double *diameters,
                          const hdmd_potential *pot, hdmd_precision prec, void *cuda_stream,
                          hdmd_system **out) {
    hdmd_system *sys = nullptr;
    if (!out) return fail(nullptr, HDMD_E_INVALID, "out is NULL");
    *out = nullptr;
    double smax = 0.0;
    int n = 1;
    {
        hdmd_status cst = check_create_args(d, N, L, diameters, pot, prec, &smax, &n);
        if (cst) return cst;
    }
    sys = new hdmd_system();
    sys->d = d;
    sys->N = N;
    sys->L = L;
    sys->pot = *pot;
    sys->prec = prec;
    sys->stream = (cudaStream_t)cuda_stream;
    sys->sigma_max = smax;
    Dev &dv = sys->dv;
    dv.d = d;
    dv.N = (int)N;
    dv.Npad = (int)((N + 63) / 64 * 64);
    dv.G = default_lanes(N);
    dv.lgG = __builtin_ctz(dv.G);
    dv.pack_sh = pack_shift(d, dv.Npad);
    dv.idx_mask = dv.pack_sh ? (uint32_t)(((uint64_t)1 << dv.pack_sh) - 1) : 0xFFFFFFFFu;
    dv.L = L;
    dv.halfL = 0.5 * L;
    dv.invL = 1.0 / L;
    dv.skin = pot->skin;
    dv.eps = pot->eps;
    dv.law = pot->kind;
    dv.eps_scale = pot->eps_scale;
    dv.morse_a = pot->kind == 1 ? pot->a : 0.0;
    dv.mie_n = pot->kind == 2 ? pot->n_mie : 0;
    dv.n = n;
    dv.ncells = 1;
    for (int k = 0; k < d; ++k) dv.ncells *= n;
    dv.Lsc = L / n;
    dv.invLsc = n / L;
    dv.Lsc_f = (float)dv.Lsc;
    dv.L_f = (float)L;
    dv.halfL_f = (float)(0.5 * L);
    dv.hmax_f = (float)(0.5 * smax);

    auto bail = [&](hdmd_status st) {
        destroy_system(sys);
        return st;
    };
    const size_t Np = dv.Npad, nd = (size_t)d * Np;
    const int RF = kRowFloats(d), RD = kRowDoubles(d);
    hdmd_status st;
#define DA2(ptr, count) do { st = dalloc(sys, &(ptr), (size_t)(count)); if (st) return bail(st); } while (0)
    DA2(dv.x0, nd); DA2(dv.dlt, nd); DA2(dv.v, nd); DA2(dv.F, nd);
    DA2(dv.sigma, Np); DA2(sys->inv_mass_store, Np); DA2(sys->st_f, nd);
    DA2(dv.img, nd); DA2(dv.id, Np);
    DA2(dv.gs0, Np * RF); DA2(dv.gs[0], Np * RF); DA2(dv.gs[1], Np * RF);
    DA2(dv.gd[0], Np * RD); DA2(dv.gd[1], Np * RD);
    DA2(dv.cell_count, dv.ncells); DA2(dv.cell_fill, dv.ncells); DA2(dv.cell_start, dv.ncells + 1);
    sys->cell_cap = dv.ncells;
    DA2(dv.cell_of, Np); DA2(dv.perm, Np); DA2(dv.cellid, Np); DA2(dv.batch_start, dv.ncells + 1);
    DA2(dv.tx, nd); DA2(dv.tv, nd); DA2(dv.tsig, Np); DA2(dv.tim, Np);
    DA2(dv.timg, nd); DA2(dv.tid, Np);
    DA2(dv.nnbr, Np);
    // most blocks any reducing kernel launches: kMaxLanes lanes per atom, kStepNT threads
    dv.maxblocks = (int)((Np * kMaxLanes + kStepNT - 1) / kStepNT);
    DA2(dv.partials, (size_t)kNRed * dv.maxblocks);
    DA2(dv.red, kNRed);
    DA2(dv.flags, 1);
    DA2(sys->st_x, nd); DA2(sys->st_v, nd); DA2(sys->st_m, Np); DA2(sys->st_sig, Np);
    DA2(sys->st_i, nd); DA2(sys->st_cnt, Np); DA2(sys->st_off, Np + 1);
    DA2(sys->snap_x0, nd); DA2(sys->snap_dlt, nd); DA2(sys->snap_v, nd); DA2(sys->snap_sig, Np);
    DA2(sys->snap_im, Np); DA2(sys->snap_img, nd); DA2(sys->snap_id, Np);
    DA2(sys->res_sync, 2 * kResMaxGrid * kResWordStride); DA2(sys->res_kin, 2 * kResMaxGrid);
#undef DA2
    sys->h_flags = (Flags *)pinned_get();
    sys->h_red = (double *)pinned_get();
    if (!sys->h_flags || !sys->h_red) {
        cudaGetLastError();
        return bail(fail(sys, HDMD_E_NOMEM, "pinned host allocation failed"));
    }
    if (cudaStreamCreateWithFlags(&sys->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sys->cap_stream2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sys->cap_stream3, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(sys, HDMD_E_CUDA, "stream creation failed"));
    }
    if (cudaMemsetAsync(dv.flags, 0, sizeof(Flags), sys->stream) != cudaSuccess ||
        cudaMemsetAsync(sys->res_sync, 0, sizeof(unsigned long long) * 2 * kResMaxGrid * kResWordStride, sys->stream) != cudaSuccess ||
        cudaMemsetAsync(dv.cell_count, 0, sizeof(int32_t) * dv.ncells, sys->stream) != cudaSuccess ||
        cudaMemsetAsync(dv.nnbr, 0, sizeof(int32_t) * Np, sys->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(sys, HDMD_E_CUDA, "initial memset failed"));
    }
    dv.inv_mass = nullptr;   // unit masses until set_state says otherwise
    st = alloc_lists(sys, initial_capacity(sys));
    if (st) return bail(st);
    // diameters in caller order (identity internal order until set_state)
    if (cudaMemcpyAsync(sys->st_sig, diameters, sizeof(double) * N, cudaMemcpyHostToDevice,
                        sys->stream) != cudaSuccess ||
        cudaMemcpyAsync(dv.sigma, sys->st_sig, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                        sys->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(sys, HDMD_E_CUDA, "diameter upload failed"));
    }
    if (cudaStreamSynchronize(sys->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(sys, HDMD_E_CUDA, "stream synchronize failed"));
    }
    *out = sys;
    return HDMD_OK;
}

hdmd_status set_state(hdmd_system *sys, const double *x, const double *v, const double *masses) {
    if (!sys) return fail(nullptr, HDMD_E_INVALID, "null system");
    if (!x) return fail(sys, HDMD_E_INVALID, "x is NULL");
    const int64_t N = sys->N;
    const int d = sys->d;
    for (int64_t a = 0; a < N * d; ++a)
        if (!std::isfinite(x[a]) || (v && !std::isfinite(v[a])))
            return fail(sys, HDMD_E_INVALID, "non-finite position or velocity");
    if (masses)
        for (int64_t i = 0; i < N; ++i)
            if (!(masses[i] > 0.0) || !std::isfinite(masses[i]))
                return fail(sys, HDMD_E_INVALID, "masses must be positive and finite");
    Dev &dv = sys->dv;
    // diameters back to caller order before the internal order is reset
    if (sys->have_state) {
        launch_export(dv, nullptr, nullptr, nullptr, nullptr, sys->st_sig, sys->stream);
        CKL(sys);
    } else {
        CK(cudaMemcpyAsync(sys->st_sig, dv.sigma, sizeof(double) * N, cudaMemcpyDeviceToDevice, sys->stream));
    }
    CK(cudaMemcpyAsync(sys->st_x, x, sizeof(double) * N * d, cudaMemcpyHostToDevice, sys->stream));
    if (v) CK(cudaMemcpyAsync(sys->st_v, v, sizeof(double) * N * d, cudaMemcpyHostToDevice, sys->stream));
    bool unit = true;
    if (masses)
        for (int64_t i = 0; i < N; ++i)
            if (masses[i] != 1.0) { unit = false; break; }
    sys->unit_mass = unit;
    if (!unit)
        CK(cudaMemcpyAsync(sys->st_m, masses, sizeof(double) * N, cudaMemcpyHostToDevice, sys->stream));
    dv.inv_mass = unit ? nullptr : sys->inv_mass_store;   // NULL: all masses 1
    const Dev d2 = dv;
    launch_import(d2, sys->st_x, v ? sys->st_v : nullptr, unit ? nullptr : sys->st_m, sys->stream);
    CKL(sys);
    launch_import_sigma(dv, sys->st_sig, sys->stream);
    CKL(sys);
    sys->have_state = true;
    free_graphs(sys);   // inv_mass pointer may have changed
    return build_forced(sys, 0);
}

hdmd_status set_diameters(hdmd_system *sys, const double *diameters) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    if (!diameters) return fail(sys, HDMD_E_INVALID, "diameters is NULL");
    double smax = 0.0;
    for (int64_t i = 0; i < sys->N; ++i) {
        if (!(diameters[i] > 0.0) || !std::isfinite(diameters[i]))
            return fail(sys, HDMD_E_INVALID, "diameters must be positive and finite");
        smax = std::max(smax, diameters[i]);
    }
    if (smax > sys->sigma_max)
        return fail(sys, HDMD_E_INVALID, "the largest diameter may not grow beyond its value at creation");
    CK(cudaMemcpyAsync(sys->st_sig, diameters, sizeof(double) * sys->N, cudaMemcpyHostToDevice, sys->stream));
    launch_import_sigma(sys->dv, sys->st_sig, sys->stream);
    CKL(sys);
    return build_forced(sys, sys->buf);
}

hdmd_status get_state(hdmd_system *sys, double *x, double *v, int32_t *img, double *f,
                      double *diameters) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    if (f && !sys->F_valid) {
        const bool fp64 = sys->prec == HDMD_FP64;
        st = ensure_rows(sys, sys->buf, !fp64, fp64);
        if (st) return st;
        st = force_only(sys, sys->buf, fp64, false);
        if (st) return st;
        sys->F_valid = true;
    }
    const int64_t nd = sys->N * sys->d;
    launch_export(sys->dv, x ? sys->st_x : nullptr, img ? sys->st_i : nullptr, v ? sys->st_v : nullptr,
                  f ? sys->st_f : nullptr, diameters ? sys->st_sig : nullptr, sys->stream);
    CKL(sys);
    if (x) CK(cudaMemcpyAsync(x, sys->st_x, sizeof(double) * nd, cudaMemcpyDeviceToHost, sys->stream));
    if (v) CK(cudaMemcpyAsync(v, sys->st_v, sizeof(double) * nd, cudaMemcpyDeviceToHost, sys->stream));
    if (img) CK(cudaMemcpyAsync(img, sys->st_i, sizeof(int32_t) * nd, cudaMemcpyDeviceToHost, sys->stream));
    if (f) CK(cudaMemcpyAsync(f, sys->st_f, sizeof(double) * nd, cudaMemcpyDeviceToHost, sys->stream));
    if (diameters)
        CK(cudaMemcpyAsync(diameters, sys->st_sig, sizeof(double) * sys->N, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    return HDMD_OK;
}

hdmd_status build_neighbors(hdmd_system *sys, int force, int *rebuilt) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    CK(cudaMemcpyAsync(&sys->h_flags->nbuilds, &sys->dv.flags->nbuilds, sizeof(int),
                       cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    const int nb0 = sys->h_flags->nbuilds;
    if (force) {
        st = build_forced(sys, sys->buf);
        if (st) return st;
    } else {
        st = clear_errors(sys);
        if (st) return st;
        launch_check_trigger(sys->dv, sys->stream);
        launch_rebuild(sys->dv, sys->buf, true, sys->stream);
        CKL(sys);
        st = read_flags(sys);
        if (st) return st;
        if (sys->h_flags->nbuilds != nb0) {
            sys->F_valid = false;
            sys->rows32_valid = sys->rows64_valid = true;
            if (sys->h_flags->error & ERR_OVERFLOW) {
                st = grow_lists(sys);
                if (st) return st;
                st = build_forced(sys, sys->buf);
                if (st) return st;
            }
        }
        st = clear_flag_field(sys, offsetof(Flags, rebuild), sizeof(int));
        if (st) return st;
    }
    CK(cudaMemcpyAsync(&sys->h_flags->nbuilds, &sys->dv.flags->nbuilds, sizeof(int),
                       cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    if (rebuilt) *rebuilt = sys->h_flags->nbuilds != nb0;
    return HDMD_OK;
}

hdmd_status get_neighbors(hdmd_system *sys, int32_t *counts, int32_t *idx, int64_t *total) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    if (!counts) return fail(sys, HDMD_E_INVALID, "counts is NULL");
    const int64_t N = sys->N;
    launch_list_export(sys->dv, sys->st_cnt, nullptr, nullptr, sys->stream);
    CKL(sys);
    CK(cudaMemcpyAsync(counts, sys->st_cnt, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    std::vector<int64_t> off(N + 1, 0);
    for (int64_t i = 0; i < N; ++i) off[i + 1] = off[i] + counts[i];
    if (total) *total = off[N];
    if (!idx || off[N] == 0) return HDMD_OK;
    if (off[N] > sys->st_idx_cap) {
        pool_free(sys->st_idx, sys->stream);
        sys->st_idx = nullptr;
        void *q = nullptr;
        if (pool_alloc(&q, sizeof(int32_t) * off[N], sys->stream) != cudaSuccess) {
            cudaGetLastError();
            sys->st_idx_cap = 0;
            return fail(sys, HDMD_E_NOMEM, "staging for get_neighbors failed");
        }
        sys->st_idx = (int32_t *)q;
        sys->st_idx_cap = off[N];
    }
    CK(cudaMemcpyAsync(sys->st_off, off.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, sys->stream));
    launch_list_export(sys->dv, nullptr, sys->st_idx, sys->st_off, sys->stream);
    CKL(sys);
    CK(cudaMemcpyAsync(idx, sys->st_idx, sizeof(int32_t) * off[N], cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    for (int64_t i = 0; i < N; ++i) std::sort(idx + off[i], idx + off[i + 1]);
    return HDMD_OK;
}

hdmd_status compute_forces(hdmd_system *sys, double *energy, double *virial) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    const bool fp64 = sys->prec == HDMD_FP64;
    st = ensure_rows(sys, sys->buf, !fp64, fp64);
    if (st) return st;
    st = force_only(sys, sys->buf, fp64, true);
    if (st) return st;
    sys->F_valid = true;
    st = read_flags(sys);
    if (st) return st;
    if (energy) *energy = 0.5 * sys->h_red[R_E];
    if (virial) *virial = 0.5 * sys->h_red[R_W];
    return check_device_errors(sys);
}

}  // extern "C"

namespace {

// nsteps in the current box, restarting from a snapshot on list overflow
hdmd_status md_fixed_box(hdmd_system *sys, int64_t nsteps, double dt, hdmd_thermo *last) {
    hdmd_status st = snapshot(sys, false);
    if (st) return st;
    const int buf0 = sys->buf;
    for (int attempt = 0; attempt < 4; ++attempt) {
        st = md_once(sys, nsteps, dt, last);
        if (st != HDMD_E_NBR_OVERFLOW) return st;
        // a build overflowed: restore the starting state, grow, and run again
        st = snapshot(sys, true);
        if (st) return st;
        st = grow_lists(sys);
        if (st) return st;
        st = build_forced(sys, buf0);
        if (st) return st;
    }
    return fail(sys, HDMD_E_NBR_OVERFLOW, "Verlet list kept overflowing during md_steps");
}

// Berendsen barostat step: positions and box side times mu, subcell grid
// recomputed (cell arrays grown when the grid grows), lists rebuilt
hdmd_status rescale_box(hdmd_system *sys, double mu) {
    Dev &dv = sys->dv;
    const double L = sys->L * mu;
    if (!(L > 2.0 * sys->sigma_max) || !std::isfinite(L))
        return fail(sys, HDMD_E_INVALID, "barostat: the box would fall below twice the largest diameter");
    int n = std::max(1, (int)std::floor(L / (sys->sigma_max + sys->pot.skin)));   // Eq. (7)
    while (n > 2 && std::pow((double)n, sys->d) > 8.0 * (double)sys->N + 4096.0) --n;
    int64_t nc = 1;
    for (int k = 0; k < sys->d; ++k) nc *= n;
    if (nc > sys->cell_cap) {
        int32_t **arrs[4] = {&dv.cell_count, &dv.cell_fill, &dv.cell_start, &dv.batch_start};
        for (auto pp : arrs) {
            void *q = nullptr;
            if (pool_alloc(&q, sizeof(int32_t) * (size_t)(nc + 1), sys->stream) != cudaSuccess) {
                cudaGetLastError();
                return fail(sys, HDMD_E_NOMEM, "barostat: subcell arrays");
            }
            auto it = std::find(sys->allocs.begin(), sys->allocs.end(), (void *)*pp);
            if (it != sys->allocs.end()) *it = q;
            else sys->allocs.push_back(q);
            pool_free(*pp, sys->stream);
            *pp = (int32_t *)q;
        }
        CK(cudaMemsetAsync(dv.cell_count, 0, sizeof(int32_t) * (size_t)nc, sys->stream));
        sys->cell_cap = nc;
    }
    launch_scale_positions(dv, mu, sys->stream);
    CKL(sys);
    sys->L = L;
    dv.L = L;
    dv.halfL = 0.5 * L;
    dv.invL = 1.0 / L;
    dv.n = n;
    dv.ncells = (int)nc;
    dv.Lsc = L / n;
    dv.invLsc = n / L;
    dv.Lsc_f = (float)dv.Lsc;
    dv.L_f = (float)L;
    dv.halfL_f = (float)(0.5 * L);
    free_graphs(sys);          // the graphs hold the box in their kernel arguments
    sys->F_valid = false;
    sys->rows32_valid = sys->rows64_valid = false;
    return build_forced(sys, sys->buf);
}

}  // namespace

extern "C" {

hdmd_status md_steps(hdmd_system *sys, int64_t nsteps, double dt, hdmd_thermo *last) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    if (nsteps < 0) return fail(sys, HDMD_E_INVALID, "nsteps must be >= 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(sys, HDMD_E_INVALID, "dt must be positive");
    if (!(sys->baro_tau > 0.0)) return md_fixed_box(sys, nsteps, dt, last);
    hdmd_thermo th{};
    int64_t left = nsteps, done = 0, rebuilds = 0;
    bool rescaled_last = false;
    while (left > 0) {
        const int64_t chunk = std::min(left, sys->baro_n - sys->baro_count);
        st = md_fixed_box(sys, chunk, dt, &th);
        if (st) return st;
        rebuilds += th.rebuilds;
        left -= chunk;
        done += chunk;
        sys->baro_count += chunk;
        rescaled_last = false;
        if (sys->baro_count == sys->baro_n) {
            const double base = 1.0 - sys->baro_beta * ((double)sys->baro_n * dt / sys->baro_tau) *
                                          (sys->baro_P - th.P);
            if (!(base > 0.0))
                return fail(sys, HDMD_E_INVALID, "barostat: the rescaling would make the box vanish");
            st = rescale_box(sys, std::pow(base, 1.0 / sys->d));
            if (st) return st;
            sys->baro_count = 0;
            rescaled_last = true;
            ++rebuilds;
        }
    }
    if (rescaled_last || nsteps == 0) {   // thermo of the (rescaled) end state
        st = md_fixed_box(sys, 0, dt, &th);
        if (st) return st;
    }
    if (last) {
        *last = th;
        last->steps = done;
        last->rebuilds = rebuilds;
    }
    return HDMD_OK;
}

hdmd_status set_barostat(hdmd_system *sys, double P_target, double tau_P, double beta,
                         int64_t n_baro) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    if (!std::isfinite(P_target) || std::isnan(tau_P))
        return fail(sys, HDMD_E_INVALID, "P_target must be finite");
    if (tau_P > 0.0 && (!(beta > 0.0) || !std::isfinite(beta) || n_baro < 1))
        return fail(sys, HDMD_E_INVALID, "barostat needs beta > 0 and n_baro >= 1");
    sys->baro_P = P_target;
    sys->baro_tau = tau_P > 0.0 && std::isfinite(tau_P) ? tau_P : 0.0;
    sys->baro_beta = beta;
    sys->baro_n = n_baro;
    sys->baro_count = 0;
    return HDMD_OK;
}

hdmd_status fire_minimize(hdmd_system *sys, const hdmd_fire_params *params, hdmd_fire_result *res) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    hdmd_fire_params p;
    if (params) {
        p = *params;
    } else {
        p.dt0 = 0.005; p.dt_max = 0.05; p.dt_min = 1e-4; p.f_inc = 1.1; p.f_dec = 0.5;
        p.alpha0 = 0.25; p.f_alpha = 0.99; p.f_tol = 1e-10; p.polish_tol = 1e-6;
        p.n_delay = 20; p.n_neg_max = 2000; p.max_iter = 1000000; p.initial_delay = 1;
        p.e_thres = 0.0; p.f_thres = 0.0; p.dx_max = 0.0;
    }
    if (!(p.e_thres >= 0) || !(p.f_thres >= 0) || !(p.dx_max >= 0) || !std::isfinite(p.e_thres) ||
        !std::isfinite(p.f_thres) || !std::isfinite(p.dx_max))
        return fail(sys, HDMD_E_INVALID, "e_thres, f_thres and dx_max must be >= 0 and finite");
    if (!(p.dt0 > 0) || !(p.dt_max >= p.dt0) || !(p.dt_min > 0) || !(p.dt_min <= p.dt0) ||
        !(p.f_inc >= 1) || !(p.f_dec > 0 && p.f_dec <= 1) || !(p.alpha0 >= 0 && p.alpha0 <= 1) ||
        !(p.f_alpha > 0 && p.f_alpha <= 1) || !(p.f_tol >= 0) || p.max_iter < 0 || p.n_delay < 0 ||
        p.n_neg_max < 0)
        return fail(sys, HDMD_E_INVALID, "invalid FIRE parameters");
    st = snapshot(sys, false);
    if (st) return st;
    for (int attempt = 0; attempt < 4; ++attempt) {
        st = fire_once(sys, p, res);
        if (st != HDMD_E_NBR_OVERFLOW) return st;
        st = snapshot(sys, true);
        if (st) return st;
        st = grow_lists(sys);
        if (st) return st;
        st = build_forced(sys, 0);
        if (st) return st;
    }
    return fail(sys, HDMD_E_NBR_OVERFLOW, "Verlet list kept overflowing during FIRE");
}

hdmd_status swap_sweep(hdmd_system *sys, int nsweeps, double T, double p, uint64_t seed,
                       const int32_t *pairs, const double *uniforms, int64_t npairs,
                       int64_t *accepted, uint8_t *accepted_flags) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    if (!(T > 0.0) || std::isnan(T)) return fail(sys, HDMD_E_INVALID, "T must be positive");
    const int64_t N = sys->N;
    int M;
    if (pairs) {
        if (!uniforms) return fail(sys, HDMD_E_INVALID, "explicit pairs need uniforms");
        if (npairs < 1 || npairs > (int64_t)1 << 26) return fail(sys, HDMD_E_INVALID, "npairs out of range");
        for (int64_t k = 0; k < npairs; ++k) {
            const int32_t i = pairs[2 * k], j = pairs[2 * k + 1];
            if (i < 0 || j < 0 || i >= N || j >= N || i == j)
                return fail(sys, HDMD_E_INVALID, "pair atoms must be distinct caller indices in [0, N)");
            if (!(uniforms[k] >= 0.0 && uniforms[k] < 1.0))
                return fail(sys, HDMD_E_INVALID, "uniforms must lie in [0, 1)");
        }
        M = (int)npairs;
        nsweeps = 1;
    } else {
        if (nsweeps < 0) return fail(sys, HDMD_E_INVALID, "nsweeps must be >= 0");
        if (!(p > 0.0 && p <= 1.0)) return fail(sys, HDMD_E_INVALID, "p must be in (0, 1]");
        M = (int)std::max<int64_t>(1, std::llround(p * (double)N));
    }
    if (nsweeps == 0) { if (accepted) *accepted = 0; return HDMD_OK; }
    st = swap_alloc(sys, M, std::max(sys->sw.scap, swap_list_estimate(sys)));
    if (st) return st;
    SwapDev &sw = sys->sw;
    sw.npairs = M;
    sw.T = T;
    sw.rcut = sys->sigma_max;
    st = ensure_rows(sys, sys->buf, true, sys->rows64_valid);
    if (st) return st;
    CK(cudaMemsetAsync(sw.nacc, 0, sizeof(unsigned long long), sys->stream));
    for (int s = 0; s < nsweeps; ++s) {
        if (pairs) {
            CK(cudaMemcpyAsync(sw.ids, pairs, sizeof(int32_t) * 2 * M, cudaMemcpyHostToDevice, sys->stream));
            CK(cudaMemcpyAsync(sw.u, uniforms, sizeof(double) * M, cudaMemcpyHostToDevice, sys->stream));
        } else {
            launch_swap_draw(sw, seed, s, (int)N, sys->stream);
            CKL(sys);
        }
        st = swap_pass(sys);
        if (st) return st;
    }
    unsigned long long nacc = 0;
    CK(cudaMemcpyAsync(&sys->h_flags->total_entries, sw.nacc, sizeof(unsigned long long), cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    nacc = (unsigned long long)sys->h_flags->total_entries;
    if (accepted) *accepted = (int64_t)nacc;
    if (accepted_flags) {
        std::vector<int8_t> stv(M);
        CK(cudaMemcpyAsync(stv.data(), sw.state, M, cudaMemcpyDeviceToHost, sys->stream));
        CK(cudaStreamSynchronize(sys->stream));
        for (int k = 0; k < M; ++k) accepted_flags[k] = stv[k] == 2;
    }
    // diameters changed: the list radii and the rows' sigma/2 are stale
    return build_forced(sys, sys->buf);
}

hdmd_status profile_kernels(hdmd_system *sys, int reps, double dt, double *ms_out) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    if (!ms_out || reps < 1 || reps > 100000 || !(dt > 0.0))
        return fail(sys, HDMD_E_INVALID, "profile_kernels: bad arguments");
    const bool fp64 = sys->prec == HDMD_FP64;
    st = ensure_rows(sys, sys->buf, !fp64, fp64);
    if (st) return st;
    if (!sys->F_valid) {
        st = force_only(sys, sys->buf, fp64, false);
        if (st) return st;
        sys->F_valid = true;
    }
    st = snapshot(sys, false);
    if (st) return st;
    const int buf0 = sys->buf;
    std::vector<cudaEvent_t> ev(2 * reps);
    for (auto &e : ev) CK(cudaEventCreate(&e));
    auto timed = [&](auto launch) -> double {
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(ev[2 * r], sys->stream);
            launch(r);
            cudaEventRecord(ev[2 * r + 1], sys->stream);
        }
        cudaStreamSynchronize(sys->stream);
        double tot = 0.0;
        for (int r = 0; r < reps; ++r) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]);
            tot += ms;
        }
        return tot / reps;
    };
    int cur = buf0;
    ms_out[0] = timed([&](int) {
        StepCfg c = base_cfg(sys, dt);
        c.compute_force = 1; c.kick2 = 1; c.kick1_drift = 1;
        c.in_buf = cur; c.out_buf = 1 - cur;
        launch_step(sys->dv, c, sys->stream);
        cur = 1 - cur;
    });
    ms_out[1] = timed([&](int) { launch_rebuild(sys->dv, cur, false, sys->stream); });
    ms_out[2] = timed([&](int) { force_only(sys, cur, fp64, false); });
    // the resident kernel: one launch of up to 20 reps steps (it stops early
    // when the trigger fires), its duration over the steps it ran
    ms_out[3] = 0.0;
    ResPlan pl;
    if (resident_plan(sys, &pl)) {
        const long long want = 20LL * reps;
        launch_set_res_left(sys->dv, want, sys->stream);
        ResCfg rc = resident_cfg(sys, pl, cur, dt);
        cudaEventRecord(ev[0], sys->stream);
        cudaError_t e = launch_md_resident(sys->dv, rc, pl.grid, pl.smem, sys->stream);
        cudaEventRecord(ev[1], sys->stream);
        if (e == cudaSuccess) {
            cudaStreamSynchronize(sys->stream);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            st = read_flags(sys);
            const long long ran = want - sys->h_flags->res_left;
            if (!st && ran > 0) ms_out[3] = (double)ms / (double)ran;
        } else {
            cudaGetLastError();
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    CKL(sys);
    st = snapshot(sys, true);
    if (st) return st;
    return build_forced(sys, buf0);
}

hdmd_status set_reference(hdmd_system *sys, const double *x_ref) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    const size_t n = (size_t)sys->N * sys->d;
    if (x_ref)
        for (size_t a = 0; a < n; ++a)
            if (!std::isfinite(x_ref[a])) return fail(sys, HDMD_E_INVALID, "non-finite reference position");
    if (!sys->obs_ref) {
        void *q = nullptr;
        if (pool_alloc(&q, sizeof(double) * n, sys->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(sys, HDMD_E_NOMEM, "reference positions");
        }
        sys->obs_ref = (double *)q;
    }
    if (x_ref) {
        CK(cudaMemcpyAsync(sys->obs_ref, x_ref, sizeof(double) * n, cudaMemcpyHostToDevice, sys->stream));
    } else {
        launch_reference(sys->dv, sys->obs_ref, sys->stream);
        CKL(sys);
    }
    CK(cudaStreamSynchronize(sys->stream));
    return HDMD_OK;
}

hdmd_status observables(hdmd_system *sys, double a_ov, int nbins, double r_max,
                        hdmd_observables *out, double *gs) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    if (!out) return fail(sys, HDMD_E_INVALID, "out is NULL");
    if (!sys->obs_ref) return fail(sys, HDMD_E_INVALID, "no reference configuration (set_reference)");
    if (nbins < 0 || nbins > 65536) return fail(sys, HDMD_E_INVALID, "nbins must be in 0..65536");
    if (nbins > 0 && (!(r_max > 0.0) || !std::isfinite(r_max)))
        return fail(sys, HDMD_E_INVALID, "r_max must be positive");
    if (!std::isfinite(a_ov)) return fail(sys, HDMD_E_INVALID, "a_ov must be finite");
    const double a = a_ov > 0.0 ? a_ov : 0.1 * sys->d;
    if (nbins > sys->obs_hist_cap) {
        pool_free(sys->obs_hist, sys->stream);
        sys->obs_hist = nullptr;
        sys->obs_hist_cap = 0;
        void *q = nullptr;
        if (pool_alloc(&q, sizeof(unsigned int) * nbins, sys->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(sys, HDMD_E_NOMEM, "G_s histogram");
        }
        sys->obs_hist = (unsigned int *)q;
        sys->obs_hist_cap = nbins;
    }
    if (nbins > 0) CK(cudaMemsetAsync(sys->obs_hist, 0, sizeof(unsigned int) * nbins, sys->stream));
    const double w = nbins > 0 ? r_max / nbins : 1.0;
    launch_observe(sys->dv, sys->obs_ref, a * a, nbins, 1.0 / w, sys->obs_hist, 1, sys->stream);
    CKL(sys);
    std::vector<unsigned int> h((size_t)std::max(nbins, 1));
    if (nbins > 0)
        CK(cudaMemcpyAsync(h.data(), sys->obs_hist, sizeof(unsigned int) * nbins, cudaMemcpyDeviceToHost,
                           sys->stream));
    st = read_flags(sys);
    if (st) return st;
    const double N = (double)sys->N, d = (double)sys->d;
    out->msd = sys->h_red[0] / N;
    out->mqd = sys->h_red[1] / N;
    out->alpha2 = out->msd > 0.0 ? d * out->mqd / ((d + 2.0) * out->msd * out->msd) - 1.0 : 0.0;
    out->f_ov = sys->h_red[2] / N;
    out->Z = sys->h_red[R_P] / N;
    if (gs)
        for (int b = 0; b < nbins; ++b) gs[b] = (double)h[b] / (N * w);
    return HDMD_OK;
}

hdmd_status set_rebuild_rule(hdmd_system *sys, int rule, int n_bet) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    if ((rule != 0 && rule != 1) || n_bet < 1)
        return fail(sys, HDMD_E_INVALID, "rule must be 0 or 1 and n_bet >= 1");
    sys->rule = rule;
    sys->n_bet = rule == 1 ? n_bet : 1;
    st = clear_flag_field(sys, offsetof(Flags, md_step), sizeof(long long));
    if (st) return st;
    free_graphs(sys);   // the step graphs hold the rule
    return HDMD_OK;
}

hdmd_status set_list_radius(hdmd_system *sys, int global) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    if (global != 0 && global != 1) return fail(sys, HDMD_E_INVALID, "global must be 0 or 1");
    sys->dv.rglobal = global ? sys->sigma_max + sys->pot.skin : 0.0;
    sys->dv.rglobal_f = (float)sys->dv.rglobal;
    free_graphs(sys);   // the graphs hold the system description
    return build_forced(sys, sys->buf);
}

hdmd_status get_box(hdmd_system *sys, double *L) {
    if (!sys) return fail(nullptr, HDMD_E_INVALID, "null system");
    if (!L) return fail(sys, HDMD_E_INVALID, "L is NULL");
    *L = sys->L;
    return HDMD_OK;
}

hdmd_status set_thermostat(hdmd_system *sys, double T_target, double tau) {
    hdmd_status st = validate_sys(sys);
    if (st) return st;
    if (!(T_target >= 0.0) || !std::isfinite(T_target) || std::isnan(tau))
        return fail(sys, HDMD_E_INVALID, "T_target must be >= 0 and finite");
    sys->nvt_T = T_target;
    sys->nvt_tau = tau > 0.0 && std::isfinite(tau) ? tau : 0.0;
    free_graphs(sys);   // the step graphs hold the thermostat constants
    return HDMD_OK;
}

hdmd_status get_info(hdmd_system *sys, hdmd_info *info) {
    if (!sys) return fail(nullptr, HDMD_E_INVALID, "null system");
    if (!info) return fail(sys, HDMD_E_INVALID, "info is NULL");
    CK(cudaMemcpyAsync(sys->h_flags, sys->dv.flags, sizeof(Flags), cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    info->d = sys->d;
    info->N = sys->N;
    info->L = sys->L;
    info->n_cell = sys->dv.n;
    info->n_cells = sys->dv.ncells;
    info->list_capacity = sys->dv.cap;
    info->lanes_per_atom = sys->dv.G;
    info->max_list_length = sys->h_flags->max_count;
    info->total_list_entries = sys->h_flags->total_entries;
    info->precision = sys->prec;
    info->graphs = sys->use_graphs && sys->graphs_ok;
    info->device_bytes = sys->bytes;
    ResPlan pl;
    info->resident = resident_plan(sys, &pl) ? pl.grid : 0;
    return HDMD_OK;
}

hdmd_status set_resident(hdmd_system *sys, int on) {
    if (!sys) return fail(nullptr, HDMD_E_INVALID, "null system");
    sys->use_resident = on ? 1 : 0;
    return HDMD_OK;
}

hdmd_status set_tuning(hdmd_system *sys, int lanes_per_atom, int use_graphs) {
    if (!sys) return fail(nullptr, HDMD_E_INVALID, "null system");
    if (lanes_per_atom) {
        if (lanes_per_atom < 1 || lanes_per_atom > 32 || (lanes_per_atom & (lanes_per_atom - 1)))
            return fail(sys, HDMD_E_INVALID, "lanes_per_atom must be a power of two in 1..32");
        sys->dv.G = lanes_per_atom;
        sys->dv.lgG = __builtin_ctz(lanes_per_atom);
        hdmd_status st = alloc_lists(sys, sys->dv.cap);
        if (st) return st;
    }
    if (use_graphs >= 0) {
        sys->use_graphs = use_graphs ? 1 : 0;
        if (use_graphs) sys->graphs_ok = true;
    }
    free_graphs(sys);
    if (sys->have_state) return build_forced(sys, sys->buf);
    return HDMD_OK;
}

hdmd_status destroy_system(hdmd_system *sys) {
    if (!sys) return HDMD_OK;
    if (sys->stream) cudaStreamSynchronize(sys->stream);
    free_graphs(sys);
    swap_free(sys);
    for (void *p : sys->allocs) pool_free(p, sys->stream);
    pool_free(sys->nbr, sys->stream);
    pool_free(sys->code, sys->stream);
    pool_free(sys->st_idx, sys->stream);
    pool_free(sys->obs_ref, sys->stream);
    pool_free(sys->obs_hist, sys->stream);
    pinned_put(sys->h_flags);
    pinned_put(sys->h_red);
    if (sys->cap_stream) cudaStreamDestroy(sys->cap_stream);
    if (sys->cap_stream2) cudaStreamDestroy(sys->cap_stream2);
    if (sys->cap_stream3) cudaStreamDestroy(sys->cap_stream3);
    cudaGetLastError();
    delete sys;
    return HDMD_OK;
}

const char *hdmd_last_error(const hdmd_system *sys) {
    if (sys) return sys->err.c_str();
    return g_thread_err.c_str();
}

}  // extern "C"
