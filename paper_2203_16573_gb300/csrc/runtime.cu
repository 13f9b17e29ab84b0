// runtime.cu -- host runtime behind include/ssx.h: context, device grids,
// the operators of the source subproblem built from stencil sweeps, the
// Algorithm 1 driver and the C ABI entry points.
//
// Operators (W. W. Symes, arXiv 2203.16573):
//   S      = Pi_0 S_{z_s,z_r} Pi_0^T              eqn:sdef (full-grid sweep)
//   S^T                                            eqn:sadj1 (reverse sweep)
//   W~_m^{-1} = -4 Pi_1 S^T J S Pi_1^T on the z_s slab   eqn:winvcomp, eqn:lamnear
//   W~_d      = same construction at z_r               eqn:wdef
//   W~_m      = -1 Pi_0 S^T J S Pi_0^T on the z_s slab  wcomp (prefactor from
//               eqn:snull2mod with the second line of eqn:approxinv)
//   J = Pi_0^T Pi_1 + Pi_1^T Pi_0 (exchange of the two trace components)
//   N = S^T W~_d S + alpha A^T W~_m A               eqn:normpart, eqn:sadjwt
//   M^{-1} = D W~_m^{-1} D, D = (I + alpha A^T A)^{-1/2}   eqn:defprecond
// The thin-slab data sit dz further along the direction from the source line
// to the receiver line; the printed prefactors hold when that direction is
// towards smaller z (the geometry of the paper's examples) and change sign in
// the mirrored geometry so that the weights stay positive.
//
// Each sweep (memsets + nt step kernels) is captured once into a CUDA graph
// per (grid, buffers) and replayed; all operators run on the context's own
// non-blocking stream, ordered against the caller's stream by events.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <type_traits>
#include <deque>
#include <functional>
#include <map>
#include <tuple>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ssx.h"
#include "ssx_internal.cuh"

using namespace ssx;

namespace {

struct DGrid {
    FieldLayout L{};
    int nx = 0, nz = 0;       // physical points of this grid
    int row0 = 0;             // model row of this grid's physical row 0
    double z_origin = 0.0;    // depth of physical row 0, km
    float *mem = nullptr;     // kap | buffer 0 (p vx vz) | buffer 1 (p vx vz)
    float *tab = nullptr;     // sponge tables: sxi sxh (NX each) szi szh (NZ each)
    float *kap = nullptr;
    float *f[2][3] = {};      // origin-offset field pointers
    unsigned *flags = nullptr;  // per-tile step counters of the persistent sweep
    int cfg[2] = {-1, -1};      // tile configuration per direction (fwd, adj), -1: not tuned
    bool pers[2] = {false, false};  // whole-sweep cooperative launch per direction
    GridArgs args{};
    bool ready = false;
};

struct EvPair {
    cudaEvent_t a = nullptr, b = nullptr;
    long long steps = 0;
    double points = 0.0;
    int tag = -1;          // row of the phase breakdown (-1: not a phase)
};

// One row of the per-phase breakdown of timed sweeps: a phase name with its
// sweep count, tile count and kernel configuration.
struct PhaseRow {
    std::string name;
    int sweeps = 0, tiles = 0, cfg = -1, chain = 0;
    double ms = 0.0;
    long long steps = 0;
};

// Kernel arguments of a phase: small phases by value, large ones in a device
// table; for the TMA-staged and the marching kernels, a table of sweeps with
// their tensor maps.
struct PhaseArgs {
    JobSet set{};
    Job *dtab = nullptr;
    TmaJob *ttab = nullptr;
    MarchJob *mtab = nullptr;
    int njobs = 0, total = 0, cap = 0;
};
// Launches [t0, t1) of a phase: the span over which the same sweeps step,
// and the arguments of those sweeps alone.
struct PhaseSeg {
    int t0 = 0, t1 = 0;
    PhaseArgs pa;
};

struct Slab {
    DGrid g;
    Line plane{}, datum{};         // lines in slab coordinates
    double z0 = 0, zd = 0;
    int ix0 = 0, n = 0;
    double *tp = nullptr, *tv = nullptr;   // datum traces [nt][n]
};

}  // namespace

struct ssx_ctx {
    ssx_grid_desc gd{};
    int R = 0;
    cudaStream_t user = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::string err;

    float *vel = nullptr;      // physical model copy [nz][nx]
    float *vmax_dev = nullptr;
    double rho = 1.0, v_max = 0.0;
    bool have_model = false, have_geom = false;

    DGrid full;
    ssx_geom_desc geom{};
    Line src{}, rec{};
    double sgn = 1.0;          // +1 in the paper's examples' geometry
    Slab ss, sr;               // z_s slab (W~_m^{-1}), z_r slab (W~_d)
    Slab sm;                   // second z_s slab for W~_m, so it can share a launch with W~_d

    // multi-sweep phases: tile configuration and device job table per phase
    struct PhaseInfo {
        int cfg = -1, T = 0;
        int chain = 0;                // launches per dependent-launch chain (0: whole span)
        std::vector<PhaseSeg> segs;   // spans of launches with the same stepping sweeps
        void *tabmem = nullptr;       // their device tables (one allocation)
    };
    std::unordered_map<std::string, PhaseInfo> phases;

    // gathers: line-shaped [nt][n_line], receiver-shaped [nt][n_rec]
    double *gbuf = nullptr;
    double *h = nullptr, *r = nullptr, *g = nullptr, *p = nullptr, *q = nullptr;
    double *tl1 = nullptr, *tl2 = nullptr, *tr1 = nullptr, *tr2 = nullptr;
    double *dist = nullptr, *dist2 = nullptr, *D = nullptr;   // [n_line]
    double D_alpha = -1.0;
    double *sc = nullptr, *partials = nullptr;                // device scalars
    double *sc_host = nullptr;                                // pinned
    std::vector<double> hostD;

    int *d_err = nullptr;      // persistent-sweep wait timeout flag (device)
    // velocity gradient: wavefield checkpoints and recompute slots (floats),
    // accumulator and trace buffers (doubles); grown on demand, kept
    float *gw = nullptr;
    size_t gw_floats = 0;
    double grad_alpha = 0.0;          // alpha of the last gradient (its Phi: 2 scalars in gwd)
    bool have_grad = false;
    double *gwd = nullptr;
    size_t gw_doubles = 0;
    int sweep_mode = SSX_SWEEP_AUTO;
    int cap[kNumTileCfgs][2];         // co-resident CTAs of the persistent kernels (-1: unknown)
    int tma_cap[kNumTileCfgs];        // co-resident CTAs of the TMA-staged phase kernel (-1: unknown)
    int march_cap[kNumMarchCfgs];     // co-resident CTAs of the marching phase kernel (-1: unknown)
    int forced_cfg = -1;              // tile configuration fixed by the caller (-1: autotune)
    bool stall_next = false;          // test hook: stall one tile of the next persistent sweep
    int hook = SSX_HOOK_NONE;         // test hook of ssx_set_test_hook and its iteration
    int hook_k = -1;
    bool use_graphs = true;
    bool log_tuning = false;          // SSX_LOG_TUNING=1: print the phase tuner's timings
    std::unordered_map<std::string, cudaGraphExec_t> graphs;
    std::unordered_map<std::string, long long> graph_nodes;
    std::unordered_map<std::string, int> key_uses;   // runs of each key not yet captured

    bool timing = false;
    std::vector<EvPair> evs;
    size_t ev_used = 0;
    ssx_stats st{};
    std::vector<PhaseRow> phase_rows;          // timed phases, in order of first appearance
    std::unordered_map<std::string, int> phase_row_of;
    int cur_tag = -1;                          // row of the phase being enqueued
};

namespace {

int fail(ssx_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(c, e_ == cudaErrorMemoryAllocation ? SSX_ERR_OOM : SSX_ERR_CUDA,  \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

#define TRY(expr)                      \
    do {                               \
        int rc_ = (expr);              \
        if (rc_ != SSX_OK) return rc_; \
    } while (0)


// Phase-kernel configuration ids: 0 .. kNumTileCfgs - 1 the plain tile kernel
// (shape id), kNumTileCfgs .. 2 kNumTileCfgs - 1 the TMA-staged tile kernel of
// shape id - kNumTileCfgs, then the marching kernel's shapes, then the
// two-step kernel's (single-sweep phases: two time steps per launch).
constexpr int kCfgMarch0 = 2 * kNumTileCfgs;
constexpr int kCfgTwo0 = kCfgMarch0 + kNumMarchCfgs;
constexpr int kNumAllCfgs = kCfgTwo0 + kNumTwoCfgs;
void tile_dims(int cfg, int *tx, int *tz) {
    const TileCfg &t = cfg >= kCfgTwo0     ? kTwoCfgs[cfg - kCfgTwo0]
                       : cfg >= kCfgMarch0 ? kMarchCfgs[cfg - kCfgMarch0]
                                           : kTileCfgs[cfg % kNumTileCfgs];
    *tx = t.tx;
    *tz = t.tz;
}

// ---------------------------------------------------------------- grids --
int grid_alloc(ssx_ctx *c, DGrid &G, int nx, int nz, int row0, double z_origin) {
    const int nsp = c->gd.n_sponge;
    G.nx = nx;
    G.nz = nz;
    G.row0 = row0;
    G.z_origin = z_origin;
    G.L = field_layout(nx + 2 * nsp, nz + 2 * nsp);
    const FieldLayout &L = G.L;
    const size_t E = L.elems();
    if (G.mem) cudaFree(G.mem);
    if (G.tab) cudaFree(G.tab);
    G.mem = nullptr;
    G.tab = nullptr;
    // kap | buffer 0 (p vx vz) | buffer 1 (p vx vz) | C_p
    CK(cudaMalloc(&G.mem, 8 * E * sizeof(float)));
    CK(cudaMalloc(&G.tab, 2 * (size_t)(L.NX + L.NZ) * sizeof(float)));
    CK(cudaMemsetAsync(G.mem, 0, 8 * E * sizeof(float), c->s));
    int max_tiles = 0;
    for (int k = 0; k < kNumTileCfgs; k++) {
        const int t = ((L.NX + kTileCfgs[k].tx - 1) / kTileCfgs[k].tx) *
                      ((L.NZ + kTileCfgs[k].tz - 1) / kTileCfgs[k].tz);
        max_tiles = t > max_tiles ? t : max_tiles;
    }
    if (G.flags) cudaFree(G.flags);
    G.flags = nullptr;
    CK(cudaMalloc(&G.flags, (size_t)max_tiles * sizeof(unsigned)));
    G.cfg[0] = G.cfg[1] = -1;
    G.kap = G.mem + L.origin();
    for (int b = 0; b < 2; b++)
        for (int f = 0; f < 3; f++) G.f[b][f] = G.mem + (1 + 3 * b + f) * E + L.origin();
    GridArgs &a = G.args;
    a.NX = L.NX;
    a.NZ = L.NZ;
    a.pitch = L.pitch;
    a.kap = G.kap;
    a.cpk = G.mem + 7 * E + L.origin();
    a.sxi = G.tab;
    a.sxh = G.tab + L.NX;
    a.szi = G.tab + 2 * L.NX;
    a.szh = G.tab + 2 * L.NX + L.NZ;
    for (int m = 0; m < kMaxR; m++) a.c[m] = kWeights[c->R][m];
    // sigma vanishes at integer positions nsp .. nsp+n-1 and half positions
    // nsp .. nsp+n-2; v points are valid up to NX-2 / NZ-2
    a.in_x0 = nsp;
    a.in_x1 = nsp + nx - 1;
    a.in_z0 = nsp;
    a.in_z1 = nsp + nz - 1;
    G.ready = false;
    return SSX_OK;
}

void grid_free(DGrid &G) {
    if (G.mem) cudaFree(G.mem);
    if (G.tab) cudaFree(G.tab);
    if (G.flags) cudaFree(G.flags);
    G.mem = nullptr;
    G.tab = nullptr;
    G.flags = nullptr;
}

int tiles_of(const DGrid &G, int cfg) {
    return ((G.L.NX + kTileCfgs[cfg].tx - 1) / kTileCfgs[cfg].tx) *
           ((G.L.NZ + kTileCfgs[cfg].tz - 1) / kTileCfgs[cfg].tz);
}

PersistArgs persist_args(ssx_ctx *c, const DGrid &G, int cfg, int nt) {
    PersistArgs pa{};
    for (int b = 0; b < 2; b++)
        for (int f = 0; f < 3; f++) pa.f[b][f] = G.f[b][f];
    pa.nt = nt;
    pa.tiles_x = (G.L.NX + kTileCfgs[cfg].tx - 1) / kTileCfgs[cfg].tx;
    pa.tiles_z = (G.L.NZ + kTileCfgs[cfg].tz - 1) / kTileCfgs[cfg].tz;
    pa.flags = G.flags;
    pa.err = c->d_err;
    pa.timeout_ns = 2000000000ull;   // 2 s per neighbour wait
    pa.stall_tile = -1;
    if (c->stall_next) {             // a wait that must run out: tile 0 never publishes
        pa.stall_tile = 0;
        pa.timeout_ns = 200000000ull;
        c->stall_next = false;
    }
    return pa;
}

// kappa dt/h field and sponge tables from the current model
int grid_fill(ssx_ctx *c, DGrid &G) {
    const ssx_grid_desc &d = c->gd;
    const int nsp = d.n_sponge;
    CK(launch_fill_kappa(G.kap, G.L, c->vel, d.nx, d.nz, nsp, G.row0, c->rho, d.dt / d.h, c->s));
    const double sdt = sponge_scale(c->v_max, nsp, d.h, d.dt);
    CK(launch_sponge_table(G.tab, G.tab + G.L.NX, G.L.NX, G.nx, nsp, sdt, c->s));
    CK(launch_sponge_table(G.tab + 2 * G.L.NX, G.tab + 2 * G.L.NX + G.L.NZ, G.L.NZ, G.nz, nsp,
                           sdt, c->s));
    G.args.cv = (float)(d.dt / (c->rho * d.h));
    CK(launch_fill_cpk(G.args, G.L, G.mem + 7 * G.L.elems(), c->s));
    G.ready = true;
    return SSX_OK;
}

int make_line(ssx_ctx *c, const DGrid &G, double z, int ix0, int n, double scale, Line *out) {
    const int nsp = c->gd.n_sponge;
    const double zeta = (z - G.z_origin) / c->gd.h + nsp;
    const int rc = line_at(zeta, G.L.NZ, G.nx, nsp, ix0, n, scale, out);
    if (rc == 1) return fail(c, SSX_ERR_ARG, "line depth outside the grid");
    if (rc == 2) return fail(c, SSX_ERR_ARG, "line columns outside the physical grid");
    return SSX_OK;
}

// Reads (and clears) the persistent-sweep timeout flag; synchronises.
int check_sweeps_quiet(ssx_ctx *c) {
    int *eh = reinterpret_cast<int *>(c->sc_host + SC_COUNT);
    CK(cudaMemcpyAsync(eh, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (*eh != 0) {
        const int code = *eh;
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->s));
        return fail(c, SSX_ERR_CUDA,
                    code == 2   ? "a phase kernel's tensor-copy wait timed out"
                    : code == 3 ? "the TMA phase kernel's shared memory is misaligned"
                                : "a persistent sweep's neighbour wait timed out");
    }
    return SSX_OK;
}

// ---------------------------------------------------------------- sweeps --
int run_cached(ssx_ctx *c, const std::string &key, long long nodes, long long steps, double points,
               const std::function<int(cudaStream_t)> &enqueue) {
    EvPair *ev = nullptr;
    if (c->timing) {
        if (c->ev_used == c->evs.size()) {
            EvPair e;
            CK(cudaEventCreate(&e.a));
            CK(cudaEventCreate(&e.b));
            c->evs.push_back(e);
        }
        ev = &c->evs[c->ev_used++];
        ev->steps = steps;
        ev->points = points;
        ev->tag = c->cur_tag;
        CK(cudaEventRecord(ev->a, c->s));
    }
    // A key's launches are captured into a graph the second time it runs:
    // work that never repeats (a batch whose set of shots changes every
    // round, a shot's set-up) is launched directly instead of being captured
    // once and thrown away.
    auto it = c->graphs.end();
    bool capture = false;
    if (c->use_graphs && !key.empty()) {
        it = c->graphs.find(key);
        if (it == c->graphs.end()) capture = ++c->key_uses[key] >= 2;
    }
    if (it != c->graphs.end() || capture) {
        if (it == c->graphs.end()) {
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
            int rc = enqueue(c->s);
            cudaError_t ec = cudaStreamEndCapture(c->s, &graph);
            if (rc != SSX_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            CK(ec);
            cudaGraphExec_t exec = nullptr;
            cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            CK(ei);
            it = c->graphs.emplace(key, exec).first;
            c->graph_nodes[key] = nodes;
            c->key_uses.erase(key);
        }
        CK(cudaGraphLaunch(it->second, c->s));
    } else {
        TRY(enqueue(c->s));
    }
    if (ev) CK(cudaEventRecord(ev->b, c->s));
    c->st.kernel_launches += nodes;
    c->st.point_updates += (long long)points;
    c->st.sweeps += 1;
    return SSX_OK;
}

std::string ptr_key(const char *tag, const void *a, const void *b, const void *d, const void *e) {
    char buf[160];
    snprintf(buf, sizeof buf, "%s:%p:%p:%p:%p", tag, a, b, d, e);
    return buf;
}

// Enqueue the step kernels of a sweep (direction adj) of `nt` steps, in
// configuration cfg: one cooperative launch (pers) or nt launches chained by
// programmatic dependent launch. The state starts in buffer 0.
int enqueue_steps(ssx_ctx *c, DGrid &G, bool adj, int cfg, bool pers, int nt, const FwdArgs &fa,
                  const AdjArgs &aa, cudaStream_t s) {
    const int R = c->R;
    if (pers) {
        if (adj)
            CK(launch_adj_persist(aa, persist_args(c, G, cfg, nt), R, cfg, s));
        else
            CK(launch_fwd_persist(fa, persist_args(c, G, cfg, nt), R, cfg, s));
        return SSX_OK;
    }
    FwdArgs a = fa;
    AdjArgs b = aa;
    for (int t = 0; t < nt; t++) {
        const int bi = t & 1, bo = bi ^ 1;
        if (adj) {
            b.p_in = G.f[bi][0];
            b.vx_in = G.f[bi][1];
            b.vz_in = G.f[bi][2];
            b.p_out = G.f[bo][0];
            b.vx_out = G.f[bo][1];
            b.vz_out = G.f[bo][2];
            b.n = nt - 1 - t;
            CK(launch_adj_step(b, R, cfg, s, true));
        } else {
            a.p_in = G.f[bi][0];
            a.vx_in = G.f[bi][1];
            a.vz_in = G.f[bi][2];
            a.p_out = G.f[bo][0];
            a.vx_out = G.f[bo][1];
            a.vz_out = G.f[bo][2];
            a.n = t;
            CK(launch_fwd_step(a, R, cfg, s, true));
        }
    }
    return SSX_OK;
}

int capacity(ssx_ctx *c, int cfg, bool adj) {
    int &cap = c->cap[cfg][adj ? 1 : 0];
    if (cap < 0) cap = persist_capacity(c->R, cfg, adj);
    return cap;
}

// Pick the tile configuration and launch form of a grid's sweeps in one
// direction by timing each admissible candidate on a short source-free sweep
// (all configurations give identical results, so only speed matters).
// Tuned choices are shared by every context of the process with a grid of the
// same shape (padded size, sponge width, order), direction and sweep mode, so
// the shots of a survey tune once.
struct TuneKey {
    int dev, NX, NZ, nsp, R, adj, mode;
    bool operator<(const TuneKey &o) const {
        return std::tie(dev, NX, NZ, nsp, R, adj, mode) <
               std::tie(o.dev, o.NX, o.NZ, o.nsp, o.R, o.adj, o.mode);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, bool>> g_tuned;

int select_config(ssx_ctx *c, DGrid &G, bool adj) {
    const int d = adj ? 1 : 0;
    if (G.cfg[d] >= 0) return SSX_OK;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    const TuneKey key{dev, G.L.NX, G.L.NZ, c->gd.n_sponge, c->R, d, c->sweep_mode};
    if (c->forced_cfg < 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            G.cfg[d] = it->second.first;
            G.pers[d] = it->second.second;
            return SSX_OK;
        }
    }
    struct Cand {
        int cfg;
        bool pers;
    };
    std::vector<Cand> cands;
    for (int k = 0; k < kNumTileCfgs; k++) {
        if (c->forced_cfg >= 0 && k != c->forced_cfg % kNumTileCfgs) continue;
        // below order 8 a quad shape runs as its strip twin: not timed twice
        if (c->forced_cfg < 0 && kTileCfgs[k].quads && c->R != kMaxR) continue;
        if (c->sweep_mode != SSX_SWEEP_PERSISTENT) cands.push_back({k, false});
        if (c->sweep_mode != SSX_SWEEP_STEP && tiles_of(G, k) <= capacity(c, k, adj))
            cands.push_back({k, true});
    }
    if (cands.empty())
        return fail(c, SSX_ERR_ARG, "no tile configuration fits the requested sweep mode");
    if (cands.size() > 1) {
        const int nt = c->gd.nt < 48 ? c->gd.nt : 48;
        FwdArgs fa{};
        AdjArgs aa{};
        fa.g = aa.g = G.args;
        fa.src = aa.src = c->src;
        fa.rec = aa.rec = c->rec;
        fa.src.n = aa.src.n = fa.rec.n = aa.rec.n = 0;   // no injection or sampling
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        float best = 1e30f;
        int bi = 0;
        for (size_t q = 0; q < cands.size(); q++) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            CK(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
            int rc = enqueue_steps(c, G, adj, cands[q].cfg, cands[q].pers, nt, fa, aa, c->s);
            cudaError_t ec = cudaStreamEndCapture(c->s, &graph);
            if (rc != SSX_OK) return rc;
            CK(ec);
            cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            CK(ei);
            float ms = 1e30f;
            for (int rep = 0; rep < 3; rep++) {
                CK(cudaMemsetAsync(G.flags, 0, (size_t)tiles_of(G, cands[q].cfg) * sizeof(unsigned), c->s));
                CK(cudaEventRecord(e0, c->s));
                CK(cudaGraphLaunch(exec, c->s));
                CK(cudaEventRecord(e1, c->s));
                CK(cudaEventSynchronize(e1));
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, e0, e1));
                if (rep > 0 && t < ms) ms = t;
            }
            cudaGraphExecDestroy(exec);
            if (ms < best) {
                best = ms;
                bi = (int)q;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        TRY(check_sweeps_quiet(c));
        G.cfg[d] = cands[bi].cfg;
        G.pers[d] = cands[bi].pers;
    } else {
        G.cfg[d] = cands[0].cfg;
        G.pers[d] = cands[0].pers;
    }
    if (c->forced_cfg < 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[key] = {G.cfg[d], G.pers[d]};
    }
    return SSX_OK;
}

// forward sweep from rest: sources on `src` -> traces on `rec`
int sim_fwd(ssx_ctx *c, DGrid &G, const Line &src, const double *hs, const double *fs,
            const Line &rec, double *outp, double *outv, bool cache = true) {
    if (!G.ready) return fail(c, SSX_ERR_ARG, "velocity model not set");
    TRY(select_config(c, G, false));
    const int nt = c->gd.nt, cfg = G.cfg[0];
    const bool pers = G.pers[0];
    auto enqueue = [&, nt, cfg, pers](cudaStream_t s) -> int {
        const size_t E = G.L.elems();
        if (outp) CK(cudaMemsetAsync(outp, 0, (size_t)nt * rec.n * sizeof(double), s));
        if (outv) CK(cudaMemsetAsync(outv, 0, (size_t)nt * rec.n * sizeof(double), s));
        CK(cudaMemsetAsync(G.mem + E, 0, 3 * E * sizeof(float), s));
        if (pers) CK(cudaMemsetAsync(G.flags, 0, (size_t)tiles_of(G, cfg) * sizeof(unsigned), s));
        FwdArgs a{};
        a.g = G.args;
        a.src = src;
        a.hsrc = hs;
        a.fsrc = fs;
        a.rec = rec;
        a.outp = outp;
        a.outv = outv;
        return enqueue_steps(c, G, false, cfg, pers, nt, a, AdjArgs{}, s);
    };
    const double pts = (double)G.L.NX * G.L.NZ * nt;
    const long long nodes = pers ? 1 : nt;
    if (!cache || pers) {
        const bool g0 = c->use_graphs;
        c->use_graphs = false;
        int rc = run_cached(c, "", nodes, nt, pts, enqueue);
        c->use_graphs = g0;
        return rc;
    }
    char tag[96];
    snprintf(tag, sizeof tag, "fwd%p:%d:%d:c%d", (void *)&G, src.kp, rec.kp, cfg);
    return run_cached(c, ptr_key(tag, hs, fs, outp, outv), nodes, nt, pts, enqueue);
}

// exact transpose of sim_fwd: adjoint data on `rec` -> adjoint sources on `src`
int sim_adj(ssx_ctx *c, DGrid &G, const Line &src, double *hb, double *fb, const Line &rec,
            const double *yp, const double *yv) {
    if (!G.ready) return fail(c, SSX_ERR_ARG, "velocity model not set");
    TRY(select_config(c, G, true));
    const int nt = c->gd.nt, cfg = G.cfg[1];
    const bool pers = G.pers[1];
    auto enqueue = [&, nt, cfg, pers](cudaStream_t s) -> int {
        const size_t E = G.L.elems();
        if (hb) CK(cudaMemsetAsync(hb, 0, (size_t)nt * src.n * sizeof(double), s));
        if (fb) CK(cudaMemsetAsync(fb, 0, (size_t)nt * src.n * sizeof(double), s));
        CK(cudaMemsetAsync(G.mem + E, 0, 3 * E * sizeof(float), s));
        if (pers) CK(cudaMemsetAsync(G.flags, 0, (size_t)tiles_of(G, cfg) * sizeof(unsigned), s));
        AdjArgs a{};
        a.g = G.args;
        a.src = src;
        a.hbar = hb;
        a.fbar = fb;
        a.rec = rec;
        a.yp = yp;
        a.yv = yv;
        a.p_in = G.f[0][0];
        a.vx_in = G.f[0][1];
        a.vz_in = G.f[0][2];
        CK(launch_adj_init(a, nt, s));
        return enqueue_steps(c, G, true, cfg, pers, nt, FwdArgs{}, a, s);
    };
    const double pts = (double)G.L.NX * G.L.NZ * nt;
    const long long nodes = (pers ? 1 : nt) + 1;
    if (pers) {
        const bool g0 = c->use_graphs;
        c->use_graphs = false;
        int rc = run_cached(c, "", nodes, nt, pts, enqueue);
        c->use_graphs = g0;
        return rc;
    }
    char tag[96];
    snprintf(tag, sizeof tag, "adj%p:%d:%d:%g:c%d", (void *)&G, src.kp, rec.kp, (double)src.scale, cfg);
    return run_cached(c, ptr_key(tag, hb, fb, yp, yv), nodes, nt, pts, enqueue);
}

// ---------------------------------------------------------------- phases --
// A phase runs several sweeps in the same launches (kernel k_multi): sweeps
// that are independent share each time step's launch, and a sweep that
// consumes another's trace gather runs in lockstep a step or two behind it.
struct Sweep {
    DGrid *G;
    bool adj;
    int offset;
    Line src, rec;
    const double *hs, *fs;       // forward sources
    double *outp, *outv;         // forward traces
    double *hb, *fb;             // transposed injections
    const double *yp, *yv;       // transposed data
    int nt;                      // time steps (0: the context's)
};

Sweep fwd_sweep(DGrid &G, const Line &src, const double *hs, const double *fs, const Line &rec,
                double *outp, double *outv, int offset = 0) {
    return Sweep{&G, false, offset, src, rec, hs, fs, outp, outv, nullptr, nullptr, nullptr, nullptr, 0};
}
Sweep adj_sweep(DGrid &G, const Line &src, double *hb, double *fb, const Line &rec,
                const double *yp, const double *yv, int offset = 0) {
    return Sweep{&G, true, offset, src, rec, nullptr, nullptr, nullptr, nullptr, hb, fb, yp, yv, 0};
}

std::vector<Job> make_jobs(const std::vector<Sweep> &sw, int cfg, bool quiet, int *total) {
    int TX = 0, TZ = 0;
    tile_dims(cfg, &TX, &TZ);   // the TMA-staged kernel tiles like the shape it is built on
    std::vector<Job> jobs(sw.size());
    int base = 0;
    for (size_t j = 0; j < sw.size(); j++) {
        const Sweep &w = sw[j];
        Job &J = jobs[j];
        memset(&J, 0, sizeof J);
        J.adj = w.adj ? 1 : 0;
        J.offset = w.offset;
        J.nt = w.nt;
        J.tiles_x = (w.G->L.NX + TX - 1) / TX;
        J.tiles = J.tiles_x * ((w.G->L.NZ + TZ - 1) / TZ);
        J.tx_shift = 0;
        while ((1LL << J.tx_shift) < J.tiles_x) J.tx_shift++;
        J.tx_mul = ((1ULL << (32 + J.tx_shift)) + (unsigned long long)J.tiles_x - 1) /
                   (unsigned long long)J.tiles_x;
        J.tile_base = base;
        base += J.tiles;
        for (int b = 0; b < 2; b++)
            for (int f = 0; f < 3; f++) J.f[b][f] = w.G->f[b][f];
        Line src = w.src, rec = w.rec;
        if (quiet) src.n = rec.n = 0;   // timing runs: no injection, no sampling
        if (w.adj) {
            J.aa.g = w.G->args;
            J.aa.src = src;
            J.aa.rec = rec;
            J.aa.hbar = w.hb;
            J.aa.fbar = w.fb;
            J.aa.yp = w.yp;
            J.aa.yv = w.yv;
        } else {
            J.fa.g = w.G->args;
            J.fa.src = src;
            J.fa.rec = rec;
            J.fa.hsrc = w.hs;
            J.fa.fsrc = w.fs;
            J.fa.outp = w.outp;
            J.fa.outv = w.outv;
        }
    }
    *total = base;
    return jobs;
}


PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// map of one field's whole storage (apron included), box bx x by floats;
// `f` points at the field's (k = 0, i = 0)
bool field_map(CUtensorMap *m, const float *f, const FieldLayout &L, int bx, int by) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dim[2] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows};
    const cuuint64_t stride[1] = {(cuuint64_t)L.pitch * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)(f - L.origin()), dim, stride, box,
               es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the marching kernel runs shape m for this context (order 8 only)
bool march_usable(ssx_ctx *c, int m) {
    if (c->R != kMaxR || m < 0 || m >= kNumMarchCfgs) return false;
    if (c->march_cap[m] < 0) c->march_cap[m] = march_capacity(m);
    return c->march_cap[m] > 0 && tensor_map_encoder() != nullptr;
}

// the two-step kernel runs a phase: one sweep from the phase's first launch,
// order 8
bool two_usable(ssx_ctx *c, const std::vector<Sweep> &sw) {
    return c->R == kMaxR && sw.size() == 1 && sw[0].offset == 0;
}

// the TMA-staged kernel runs shape `base` for this context (order 8 only)
bool tma_usable(ssx_ctx *c, int base) {
    if (c->R != kMaxR || base < 0 || base >= kNumTileCfgs || !tma_shape_supported(base)) return false;
    if (c->tma_cap[base] < 0) c->tma_cap[base] = tma_capacity(base);
    return c->tma_cap[base] > 0 && tensor_map_encoder() != nullptr;
}

// tensor maps of one sweep for the marching kernel of shape m: boxes of one
// block of kMarchB rows -- p and C_p over the tile with a 2k column halo, v_x
// with a k halo, v_z and kappa over the tile
bool march_job(const Sweep &w, const Job &job, int m, MarchJob *out) {
    const int TX = kMarchCfgs[m].tx, R = kMaxR, B = kMarchB;
    memset(out, 0, sizeof(MarchJob));
    out->job = job;
    const DGrid &G = *w.G;
    bool ok = true;
    for (int b = 0; b < 2; b++) {
        ok = ok && field_map(&out->map[b], G.f[b][0], G.L, TX + 4 * R, B);
        ok = ok && field_map(&out->map[2 + b], G.f[b][1], G.L, TX + 2 * R, B);
        ok = ok && field_map(&out->map[4 + b], G.f[b][2], G.L, TX, B);
    }
    ok = ok && field_map(&out->map[6], G.args.kap, G.L, TX, B);
    ok = ok && field_map(&out->map[7], G.args.cpk, G.L, TX + 4 * R, B);
    return ok;
}

// tensor maps of one sweep for the TMA-staged kernel of shape `base`: boxes
// of the tile with its halos
bool tma_job(const Sweep &w, const Job &job, int base, TmaJob *out) {
    const int TX = kTileCfgs[base].tx, TZ = kTileCfgs[base].tz, R = kMaxR;
    memset(out, 0, sizeof(TmaJob));
    out->job = job;
    const DGrid &G = *w.G;
    bool ok = true;
    for (int b = 0; b < 2; b++) {
        ok = ok && field_map(&out->map[b], G.f[b][0], G.L, TX + 4 * R, TZ + 4 * R);
        ok = ok && field_map(&out->map[2 + b], G.f[b][1], G.L, TX + 2 * R, TZ);
        ok = ok && field_map(&out->map[4 + b], G.f[b][2], G.L, TX, TZ + 2 * R - 1);
    }
    ok = ok && (job.adj ? field_map(&out->map[6], G.args.cpk, G.L, TX + 4 * R, TZ + 4 * R)
                        : field_map(&out->map[6], G.args.kap, G.L, TX, TZ));
    return ok;
}

// Kernel arguments of a set of sweeps in configuration cfg, with any device
// table appended to `host` at a 128-byte aligned offset (recorded in the
// PhaseArgs pointer fields as an offset until the table is uploaded).
int stage_args(ssx_ctx *c, const std::vector<Sweep> &sw, int cfg, bool quiet, PhaseArgs *pa,
               std::vector<unsigned char> &host) {
    std::vector<Job> jobs = make_jobs(sw, cfg, quiet, &pa->total);
    pa->njobs = (int)jobs.size();
    pa->dtab = nullptr;
    pa->ttab = nullptr;
    pa->mtab = nullptr;
    auto append = [&](const void *src, size_t bytes) -> size_t {
        const size_t off = (host.size() + 127) / 128 * 128;
        host.resize(off + bytes);
        memcpy(host.data() + off, src, bytes);
        return off;
    };
    // offsets are kept +1 in the pointer fields until the upload resolves them
    auto tag = [](size_t off) { return (void *)(off + 1); };
    if (cfg >= kCfgTwo0) {
        if (!two_usable(c, sw)) return fail(c, SSX_ERR_ARG, "two-step kernel not available");
        memset(&pa->set, 0, sizeof pa->set);
        pa->set.njobs = 1;
        pa->set.job[0] = jobs[0];
        return SSX_OK;
    }
    if (cfg >= kCfgMarch0) {
        const int m = cfg - kCfgMarch0;
        // the choice may come from another context's tuning: this context's
        // grid cap is looked up here if it is not known yet
        if (!march_usable(c, m)) return fail(c, SSX_ERR_ARG, "marching kernel not available");
        std::vector<MarchJob> mj(jobs.size());
        for (size_t j = 0; j < jobs.size(); j++)
            if (!march_job(sw[j], jobs[j], m, &mj[j])) return fail(c, SSX_ERR_CUDA, "tensor map encoding failed");
        pa->mtab = (MarchJob *)tag(append(mj.data(), mj.size() * sizeof(MarchJob)));
        pa->cap = c->march_cap[m];
        return SSX_OK;
    }
    if (cfg >= kNumTileCfgs) {
        const int base = cfg - kNumTileCfgs;
        if (!tma_usable(c, base)) return fail(c, SSX_ERR_ARG, "TMA-staged kernel not available");
        std::vector<TmaJob> tj(jobs.size());
        for (size_t j = 0; j < jobs.size(); j++)
            if (!tma_job(sw[j], jobs[j], base, &tj[j])) return fail(c, SSX_ERR_CUDA, "tensor map encoding failed");
        pa->ttab = (TmaJob *)tag(append(tj.data(), tj.size() * sizeof(TmaJob)));
        pa->cap = c->tma_cap[base];
        return SSX_OK;
    }
    if (jobs.size() <= (size_t)kMaxJobs) {
        memset(&pa->set, 0, sizeof pa->set);
        pa->set.njobs = pa->njobs;
        for (size_t j = 0; j < jobs.size(); j++) pa->set.job[j] = jobs[j];
        return SSX_OK;
    }
    pa->dtab = (Job *)tag(append(jobs.data(), jobs.size() * sizeof(Job)));
    return SSX_OK;
}

// upload the tables staged by stage_args (one allocation, one copy) and turn
// the recorded offsets into device pointers
int upload_args(ssx_ctx *c, const std::vector<unsigned char> &host, std::vector<PhaseArgs *> args,
                void **mem) {
    *mem = nullptr;
    if (host.empty()) return SSX_OK;
    CK(cudaMalloc(mem, host.size()));
    CK(cudaMemcpyAsync(*mem, host.data(), host.size(), cudaMemcpyHostToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
    unsigned char *base = (unsigned char *)*mem;
    auto fix = [&](auto *&ptr) {
        if (ptr) ptr = reinterpret_cast<std::remove_reference_t<decltype(ptr)>>(base + ((size_t)ptr - 1));
    };
    for (PhaseArgs *pa : args) {
        fix(pa->dtab);
        fix(pa->ttab);
        fix(pa->mtab);
    }
    return SSX_OK;
}

// Kernel arguments of a phase in one set (the tuner's short runs); *mem
// receives the device table, if any, for the caller to free.
int phase_args(ssx_ctx *c, const std::vector<Sweep> &sw, int cfg, bool quiet, PhaseArgs *pa,
               void **mem) {
    std::vector<unsigned char> host;
    TRY(stage_args(c, sw, cfg, quiet, pa, host));
    return upload_args(c, host, {pa}, mem);
}

int phase_len(const std::vector<Sweep> &sw) {
    int T = 0;
    for (const Sweep &w : sw) T = std::max(T, w.offset + w.nt);
    return T;
}

// the launches of a phase: transposed sweeps get their initial state (the
// transposed sampling of their last data sample) just before their first step
// Launches t0 .. t1-1 of a phase. Consecutive launches are chained by
// programmatic dependent launch, except every `chain`-th (chain > 0), which
// is an ordinary launch: on a long chain the CTAs of the next launches become
// resident early and spread unevenly over the SMs, and a launch with fewer
// tiles than SMs then runs slower per step (measured; the phase tuner picks
// the chain length).
int enqueue_launches(ssx_ctx *c, const std::vector<Sweep> &sw, const PhaseArgs &pa, int t0, int t1,
                     int cfg, cudaStream_t s, bool with_init, bool stall = false, int chain = 0) {
    // transposed sweeps starting at launch t get their initial state first
    auto inits = [&](int t) -> int {
        if (with_init)
            for (const Sweep &w : sw)
                if (w.adj && w.offset == t) {
                    AdjArgs a{};
                    a.g = w.G->args;
                    a.rec = w.rec;
                    a.yp = w.yp;
                    a.yv = w.yv;
                    a.p_in = w.G->f[0][0];
                    a.vx_in = w.G->f[0][1];
                    a.vz_in = w.G->f[0][2];
                    CK(launch_adj_init(a, w.nt, s));
                }
        return SSX_OK;
    };
    if (cfg >= kCfgTwo0) {   // two time steps per launch: launch u runs steps 2u and 2u + 1
        const int u0 = t0 / 2;
        for (int u = u0; 2 * u < t1; u++) {
            const bool brk = chain > 0 && (u - u0) % chain == 0;
            TRY(inits(2 * u));
            CK(launch_two(pa.set, pa.total, u, 2 * u + 1 < t1, cfg - kCfgTwo0, s, u != u0 && !brk));
        }
        return SSX_OK;
    }
    for (int t = t0; t < t1; t++) {
        const bool brk = chain > 0 && (t - t0) % chain == 0;
        TRY(inits(t));
        if (pa.mtab)
            CK(launch_march(pa.mtab, pa.njobs, pa.total, t, cfg - kCfgMarch0, pa.cap, c->d_err,
                            stall && t == 0 ? 200000000ull : 2000000000ull,
                            stall && t == 0 ? 0 : -1, s, !brk));
        else if (pa.ttab)
            CK(launch_multi_tma(pa.ttab, pa.njobs, pa.total, t, cfg - kNumTileCfgs, pa.cap, c->d_err,
                                stall && t == 0 ? 200000000ull : 2000000000ull,
                                stall && t == 0 ? 0 : -1, s, !brk));
        else if (pa.dtab)
            CK(launch_multi_tab(pa.dtab, pa.njobs, pa.total, t, c->R, cfg, s, !brk));
        else   // the span's first launch is not a dependent launch: its sweeps
               // may read their injected gathers before the grid dependency wait
            CK(launch_multi(pa.set, pa.total, t, c->R, cfg, s, t != t0 && !brk));
    }
    return SSX_OK;
}

// Phase tuning results, shared by every context of the process: phases of up
// to kMaxJobs sweeps by their exact shape (each sweep's padded grid,
// direction and lockstep offset), larger ones (batches, whose set of shots a
// server changes every few rounds) by size class -- sweep count, total points
// (half octaves) and direction mix -- so that a batch of a new composition
// reuses the choice of one of similar size instead of timing every
// configuration again. All configurations give identical results.
std::mutex g_phase_mu;
struct PhaseChoice {
    int cfg, chain;
};
std::map<std::vector<long long>, PhaseChoice> g_phase_tuned;

std::vector<long long> phase_signature(ssx_ctx *c, const std::vector<Sweep> &sw) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<long long> k{dev, c->R, c->sweep_mode, (long long)sw.size()};
    if (sw.size() <= (size_t)kMaxJobs) {
        for (const Sweep &w : sw) {
            k.push_back(w.G->L.NX);
            k.push_back(w.G->L.NZ);
            k.push_back(w.adj);
            k.push_back(w.offset);
        }
        return k;
    }
    double pts = 0;
    int nadj = 0;
    for (const Sweep &w : sw) {
        pts += (double)w.G->L.NX * w.G->L.NZ;
        nadj += w.adj ? 1 : 0;
    }
    k[3] = -(long long)std::ceil(std::log2((double)sw.size()));
    k.push_back((long long)std::floor(2.0 * std::log2(pts)));
    k.push_back(nadj == 0 ? 0 : nadj == (int)sw.size() ? 2 : 1);
    return k;
}

// Device time of T launches of a phase in configuration cfg (a graph of the
// source-free launches, run three times, the best of the last two): 0 and
// *ok = false if the configuration cannot be set up for these sweeps.
int time_phase(ssx_ctx *c, const std::vector<Sweep> &sw, int cfg, int T, int chain, float *ms,
               int *tiles, bool *ok) {
    *ok = false;
    *ms = 1e30f;
    PhaseArgs pa;
    void *tmem = nullptr;
    if (phase_args(c, sw, cfg, true, &pa, &tmem) != SSX_OK) {   // a candidate that cannot be set up
        if (tmem) cudaFree(tmem);
        return SSX_OK;
    }
    *tiles = pa.total;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = SSX_OK;
    cudaError_t ec = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal);
    if (ec == cudaSuccess) {
        rc = enqueue_launches(c, sw, pa, 0, T, cfg, c->s, false, false, chain);
        ec = cudaStreamEndCapture(c->s, &graph);
    }
    if (rc == SSX_OK && ec == cudaSuccess) {
        ec = cudaGraphInstantiate(&exec, graph, 0);
        if (ec == cudaSuccess) ec = cudaEventCreate(&e0);
        if (ec == cudaSuccess) ec = cudaEventCreate(&e1);
        for (int rep = 0; rep < 3 && ec == cudaSuccess; rep++) {
            ec = cudaEventRecord(e0, c->s);
            if (ec == cudaSuccess) ec = cudaGraphLaunch(exec, c->s);
            if (ec == cudaSuccess) ec = cudaEventRecord(e1, c->s);
            if (ec == cudaSuccess) ec = cudaEventSynchronize(e1);
            float t = 0.f;
            if (ec == cudaSuccess) ec = cudaEventElapsedTime(&t, e0, e1);
            if (ec == cudaSuccess && rep > 0) *ms = std::min(*ms, t);
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (exec) cudaGraphExecDestroy(exec);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (tmem) cudaFree(tmem);
    if (rc != SSX_OK) return rc;
    CK(ec);
    *ok = true;
    return SSX_OK;
}

// Tile configuration of a phase: each admissible one timed on a short
// source-free run (48 launches); then the length of its dependent-launch
// chains, timed over up to 256 launches of the chosen configuration (a
// break every 8, 16 or 32 launches, or none), kept only where it gains
// more than 2 %.
int tune_phase(ssx_ctx *c, const char *name, const std::vector<Sweep> &sw, int *best_cfg,
               int *best_chain) {
    *best_chain = 0;
    const std::vector<long long> sig = phase_signature(c, sw);
    const bool forced = c->forced_cfg >= 0;
    if (forced) {
        const int f = c->forced_cfg;
        if (f >= kCfgTwo0) *best_cfg = two_usable(c, sw) ? f : 0;
        else if (f >= kCfgMarch0) *best_cfg = march_usable(c, f - kCfgMarch0) ? f : 0;
        else *best_cfg = (f >= kNumTileCfgs && !tma_usable(c, f - kNumTileCfgs)) ? f - kNumTileCfgs : f;
    } else {
        std::lock_guard<std::mutex> lock(g_phase_mu);
        auto it = g_phase_tuned.find(sig);
        if (it != g_phase_tuned.end()) {
            *best_cfg = it->second.cfg;
            *best_chain = it->second.chain;
            return SSX_OK;
        }
    }
    if (!forced) {
        const int T = std::min(phase_len(sw), 48);
        float best = 1e30f;
        for (int k = 0; k < kNumAllCfgs; k++) {
            if (k >= kCfgTwo0) {
                if (!two_usable(c, sw)) continue;
            } else if (k >= kCfgMarch0) {
                if (!march_usable(c, k - kCfgMarch0)) continue;
            } else if (k >= kNumTileCfgs && !tma_usable(c, k - kNumTileCfgs)) {
                continue;
            } else if (kTileCfgs[k % kNumTileCfgs].quads && c->R != kMaxR) {
                continue;   // below order 8 a quad shape runs as its strip twin
            }
            float ms = 0.f;
            int tiles = 0;
            bool ok = false;
            TRY(time_phase(c, sw, k, T, 0, &ms, &tiles, &ok));
            if (!ok) continue;
            if (c->log_tuning)
                std::fprintf(stderr, "ssx tune: phase %s (%zu sweeps, %d tiles) config %d: %.3f us/step\n",
                             name, sw.size(), tiles, k, 1000.0 * ms / T);
            if (ms < best) {
                best = ms;
                *best_cfg = k;
            }
        }
    }
    const int T2 = std::min(phase_len(sw), 256);
    if (T2 >= 128) {
        const int chains[] = {0, 8, 16, 32};
        float t0 = 0.f;
        for (int chain : chains) {
            float ms = 0.f;
            int tiles = 0;
            bool ok = false;
            TRY(time_phase(c, sw, *best_cfg, T2, chain, &ms, &tiles, &ok));
            if (!ok) break;
            if (c->log_tuning)
                std::fprintf(stderr, "ssx tune: phase %s config %d chain %d: %.3f us/step\n", name,
                             *best_cfg, chain, 1000.0 * ms / T2);
            if (chain == 0) t0 = ms;
            else if (ms < 0.98f * t0 && (*best_chain == 0 || ms < t0)) {
                t0 = ms;
                *best_chain = chain;
            }
        }
    }
    if (!forced) {
        std::lock_guard<std::mutex> lock(g_phase_mu);
        g_phase_tuned[sig] = PhaseChoice{*best_cfg, *best_chain};
    }
    return SSX_OK;
}

int run_phase(ssx_ctx *c, const char *name, std::vector<Sweep> sw) {
    for (Sweep &w : sw) {
        if (!w.G->ready) return fail(c, SSX_ERR_ARG, "velocity model not set");
        if (w.nt == 0) w.nt = c->gd.nt;
    }
    std::string key = name;
    for (const Sweep &w : sw) {
        char b[200];
        snprintf(b, sizeof b, "|%p%d%d:%d:%d:%d:%g:%p:%p:%p:%p:%p:%p:%p:%p", (void *)w.G, w.adj,
                 w.offset, w.nt, w.src.kp, w.rec.kp, (double)w.src.scale, (const void *)w.hs,
                 (const void *)w.fs, (void *)w.outp, (void *)w.outv, (void *)w.hb, (void *)w.fb,
                 (const void *)w.yp, (const void *)w.yv);
        key += b;
    }
    auto it = c->phases.find(key);
    if (it == c->phases.end()) {
        ssx_ctx::PhaseInfo info;
        TRY(tune_phase(c, name, sw, &info.cfg, &info.chain));
        TRY(check_sweeps_quiet(c));
        // The phase's launches split where a sweep starts or ends: each span
        // launches only the sweeps that step in it (a batch whose shots have
        // different step counts launches no CTAs for finished sweeps).
        std::vector<int> bounds;
        for (const Sweep &w : sw) {
            bounds.push_back(w.offset);
            bounds.push_back(w.offset + w.nt);
        }
        std::sort(bounds.begin(), bounds.end());
        bounds.erase(std::unique(bounds.begin(), bounds.end()), bounds.end());
        std::vector<unsigned char> host;
        for (size_t q = 0; q + 1 < bounds.size(); q++) {
            std::vector<Sweep> sub;
            for (const Sweep &w : sw)
                if (w.offset <= bounds[q] && bounds[q] < w.offset + w.nt) sub.push_back(w);
            if (sub.empty()) continue;
            PhaseSeg seg;
            seg.t0 = bounds[q];
            seg.t1 = bounds[q + 1];
            TRY(stage_args(c, sub, info.cfg, false, &seg.pa, host));
            info.segs.push_back(seg);
        }
        std::vector<PhaseArgs *> args;
        for (PhaseSeg &seg : info.segs) args.push_back(&seg.pa);
        TRY(upload_args(c, host, args, &info.tabmem));
        info.T = phase_len(sw);
        it = c->phases.emplace(key, std::move(info)).first;
    }
    const ssx_ctx::PhaseInfo &info = it->second;
    // test hook: the next TMA-staged phase withholds the copies of its first
    // tile in its first launch (run uncached, so no graph keeps the stall)
    const bool stall = c->stall_next && info.cfg >= kNumTileCfgs && info.cfg < kCfgTwo0;
    if (stall) c->stall_next = false;
    auto enqueue = [&](cudaStream_t s) -> int {
        for (const Sweep &w : sw) {
            const size_t E = w.G->L.elems();
            const size_t nr = (size_t)w.nt * w.rec.n * sizeof(double);
            const size_t ns = (size_t)w.nt * w.src.n * sizeof(double);
            if (w.outp) CK(cudaMemsetAsync(w.outp, 0, nr, s));
            if (w.outv) CK(cudaMemsetAsync(w.outv, 0, nr, s));
            if (w.hb) CK(cudaMemsetAsync(w.hb, 0, ns, s));
            if (w.fb) CK(cudaMemsetAsync(w.fb, 0, ns, s));
            CK(cudaMemsetAsync(w.G->mem + E, 0, 3 * E * sizeof(float), s));
        }
        for (const PhaseSeg &seg : info.segs)
            TRY(enqueue_launches(c, sw, seg.pa, seg.t0, seg.t1, info.cfg, s, true, stall, info.chain));
        return SSX_OK;
    };
    double pts = 0;
    long long inits = 0;
    for (const Sweep &w : sw) {
        pts += (double)w.G->L.NX * w.G->L.NZ * w.nt;
        inits += w.adj ? 1 : 0;
    }
    c->st.sweeps += (long long)sw.size() - 1;   // run_cached counts one
    if (c->timing) {   // the phase's row of the timing breakdown
        int tiles = 0;
        for (const PhaseSeg &seg : info.segs) tiles = std::max(tiles, seg.pa.total);
        const std::string rk = std::string(name) + "|" + std::to_string(sw.size()) + "|" +
                               std::to_string(tiles) + "|" + std::to_string(info.cfg) + "|" +
                               std::to_string(info.chain);
        auto r = c->phase_row_of.find(rk);
        if (r == c->phase_row_of.end()) {
            PhaseRow row;
            row.name = name;
            row.sweeps = (int)sw.size();
            row.tiles = tiles;
            row.cfg = info.cfg;
            row.chain = info.chain;
            c->phase_rows.push_back(row);
            r = c->phase_row_of.emplace(rk, (int)c->phase_rows.size() - 1).first;
        }
        c->cur_tag = r->second;
    }
    struct TagReset {
        ssx_ctx *c;
        ~TagReset() { c->cur_tag = -1; }
    } tag_reset{c};
    if (stall) {
        const bool g0 = c->use_graphs;
        c->use_graphs = false;
        const int rc = run_cached(c, "", info.T + inits, info.T, pts, enqueue);
        c->use_graphs = g0;
        return rc;
    }
    // kernel launches: one per time step, or one per two for the two-step kernel
    const long long launches = info.cfg >= kCfgTwo0 ? (info.T + 1) / 2 : info.T;
    return run_cached(c, "phase" + std::to_string(info.cfg) + key, launches + inits, info.T, pts,
                      enqueue);
}

bool fused(ssx_ctx *c) { return c->sweep_mode != SSX_SWEEP_PERSISTENT; }

// ------------------------------------------------------------- operators --
int op_S(ssx_ctx *c, const double *in, double *out) {
    if (!fused(c)) return sim_fwd(c, c->full, c->src, in, nullptr, c->rec, out, nullptr);
    return run_phase(c, "S", {fwd_sweep(c->full, c->src, in, nullptr, c->rec, out, nullptr)});
}
int op_ST(ssx_ctx *c, const double *in, double *out) {
    if (!fused(c)) return sim_adj(c, c->full, c->src, out, nullptr, c->rec, in, nullptr);
    return run_phase(c, "ST", {adj_sweep(c->full, c->src, out, nullptr, c->rec, in, nullptr)});
}
// -4 Pi_1 S^T J S Pi_1^T on a slab (eqn:winvcomp): velocity injection on the
// plane, both traces at the datum, exchanged, transposed sweep
Line scaled(const Line &l, double f) {
    Line o = l;
    o.scale = (float)f;
    return o;
}
int op_sym_lambda(ssx_ctx *c, Slab &sl, const double *in, double *out) {
    const Line pl = scaled(sl.plane, -4.0 * c->sgn);
    if (!fused(c)) {
        TRY(sim_fwd(c, sl.g, sl.plane, nullptr, in, sl.datum, sl.tp, sl.tv));
        return sim_adj(c, sl.g, pl, nullptr, out, sl.datum, sl.tv, sl.tp);
    }
    TRY(run_phase(c, "Lf", {fwd_sweep(sl.g, sl.plane, nullptr, in, sl.datum, sl.tp, sl.tv)}));
    return run_phase(c, "La", {adj_sweep(sl.g, pl, nullptr, out, sl.datum, sl.tv, sl.tp)});
}
// -Pi_0 S^T J S Pi_0^T on the z_s slab (wcomp)
int op_Wm(ssx_ctx *c, const double *in, double *out) {
    Slab &sl = c->sm;
    const Line pl = scaled(sl.plane, -1.0 * c->sgn);
    if (!fused(c)) {
        TRY(sim_fwd(c, sl.g, sl.plane, in, nullptr, sl.datum, sl.tp, sl.tv));
        return sim_adj(c, sl.g, pl, out, nullptr, sl.datum, sl.tv, sl.tp);
    }
    TRY(run_phase(c, "Mf", {fwd_sweep(sl.g, sl.plane, in, nullptr, sl.datum, sl.tp, sl.tv)}));
    return run_phase(c, "Ma", {adj_sweep(sl.g, pl, out, nullptr, sl.datum, sl.tv, sl.tp)});
}
int op_W(ssx_ctx *c, int which, const double *in, double *out) {
    switch (which) {
        case SSX_W_D: return op_sym_lambda(c, c->sr, in, out);
        case SSX_W_M: return op_Wm(c, in, out);
        case SSX_W_M_INV: return op_sym_lambda(c, c->ss, in, out);
        default: return fail(c, SSX_ERR_ARG, "unknown weight operator");
    }
}

// Lambda~ (eqn:lamtilde) or its transpose (eqn:lamtransp) on the z_s slab:
// velocity injection of r, one datum trace taken back through the other
// trace's transposed injection, -8 (orientation sign as for the weights).
int op_lambda(ssx_ctx *c, bool transpose, const double *in, double *out) {
    Slab &sl = c->ss;
    const Line pl = scaled(sl.plane, -8.0 * c->sgn);
    if (!fused(c)) {
        TRY(sim_fwd(c, sl.g, sl.plane, nullptr, in, sl.datum, sl.tp, sl.tv));
        return transpose ? sim_adj(c, sl.g, pl, nullptr, out, sl.datum, sl.tv, nullptr)
                         : sim_adj(c, sl.g, pl, nullptr, out, sl.datum, nullptr, sl.tp);
    }
    TRY(run_phase(c, "Lf", {fwd_sweep(sl.g, sl.plane, nullptr, in, sl.datum, sl.tp, sl.tv)}));
    return transpose ? run_phase(c, "LTa", {adj_sweep(sl.g, pl, nullptr, out, sl.datum, sl.tv, nullptr)})
                     : run_phase(c, "LNa", {adj_sweep(sl.g, pl, nullptr, out, sl.datum, nullptr, sl.tp)});
}

// 4 (V+_{zs,zr})^T d (eqn:approxinv): the data as a vertical load at the
// receivers, one transposed sweep, the velocity-injection read-out on z_s
int op_trinv(ssx_ctx *c, const double *d, double *h) {
    const Line sl = scaled(c->src, 4.0);
    if (!fused(c)) return sim_adj(c, c->full, sl, nullptr, h, c->rec, nullptr, d);
    return run_phase(c, "TR", {adj_sweep(c->full, sl, nullptr, h, c->rec, nullptr, d)});
}

int set_D(ssx_ctx *c, double alpha) {
    if (c->D_alpha == alpha) return SSX_OK;
    const int n = c->geom.n_line;
    c->hostD.resize(n);
    for (int j = 0; j < n; j++) {
        const double x = (c->geom.ix_line0 + j) * c->gd.h - c->geom.x_s;
        c->hostD[j] = 1.0 / std::sqrt(1.0 + alpha * x * x);
    }
    CK(cudaMemcpyAsync(c->D, c->hostD.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
    c->D_alpha = alpha;
    return SSX_OK;
}

// g = D W~_m^{-1} D r (eqn:defprecond); identity for plain CG
int op_Minv(ssx_ctx *c, int mode, double alpha, const double *r, double *g) {
    const int nt = c->gd.nt, nl = c->geom.n_line;
    if (mode == SSX_MODE_CG) {
        CK(cudaMemcpyAsync(g, r, (size_t)nt * nl * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
        return SSX_OK;
    }
    TRY(set_D(c, alpha));
    CK(launch_colscale(c->tl1, r, c->D, nt, nl, c->s));
    TRY(op_sym_lambda(c, c->ss, c->tl1, c->tl2));
    CK(launch_colscale(g, c->tl2, c->D, nt, nl, c->s));
    c->st.kernel_launches += 2;
    return SSX_OK;
}

// q = N p (eqn:normpart) or the Euclidean normal operator. Fused: phase 1
// runs S p, the W~_d slab's forward sweep one step behind it (it consumes
// S p sample n - 1) and, for alpha > 0, W~_m's forward sweep on A p; phase 2
// runs the W~_d slab's transposed sweep, S^T two steps behind it (it needs the
// slab's output sample m - 1 at the end of its reverse step m) and W~_m's
// transposed sweep.
int op_N(ssx_ctx *c, int mode, double alpha, const double *p, double *q) {
    const int nt = c->gd.nt, nl = c->geom.n_line;
    if (alpha != 0.0 && mode == SSX_MODE_PCG) {
        CK(launch_colscale(c->tl1, p, c->dist, nt, nl, c->s));
        c->st.kernel_launches += 1;
    }
    if (mode == SSX_MODE_PCG && fused(c)) {
        Slab &r = c->sr, &m = c->sm;
        std::vector<Sweep> ph1 = {fwd_sweep(c->full, c->src, p, nullptr, c->rec, c->tr1, nullptr),
                                  fwd_sweep(r.g, r.plane, nullptr, c->tr1, r.datum, r.tp, r.tv, 1)};
        std::vector<Sweep> ph2 = {adj_sweep(r.g, scaled(r.plane, -4.0 * c->sgn), nullptr, c->tr2,
                                            r.datum, r.tv, r.tp),
                                  adj_sweep(c->full, c->src, q, nullptr, c->rec, c->tr2, nullptr, 2)};
        if (alpha != 0.0) {
            ph1.push_back(fwd_sweep(m.g, m.plane, c->tl1, nullptr, m.datum, m.tp, m.tv));
            ph2.push_back(adj_sweep(m.g, scaled(m.plane, -1.0 * c->sgn), c->tl2, nullptr, m.datum,
                                    m.tv, m.tp));
        }
        TRY(run_phase(c, "N1", ph1));
        TRY(run_phase(c, "N2", ph2));
    } else {
        TRY(op_S(c, p, c->tr1));
        if (mode == SSX_MODE_PCG) {
            TRY(op_sym_lambda(c, c->sr, c->tr1, c->tr2));
            TRY(op_ST(c, c->tr2, q));
            if (alpha != 0.0) TRY(op_Wm(c, c->tl1, c->tl2));
        } else {
            TRY(op_ST(c, c->tr1, q));
        }
    }
    if (alpha != 0.0) {
        if (mode == SSX_MODE_PCG)
            CK(launch_colscale_add(q, c->tl2, c->dist, alpha, nt, nl, c->s));
        else
            CK(launch_colscale_add(q, p, c->dist2, alpha, nt, nl, c->s));
        c->st.kernel_launches += 1;
    }
    return SSX_OK;
}

// ------------------------------------------------------------- plumbing --
int enter(ssx_ctx *c) {
    CK(cudaEventRecord(c->ev_in, c->user));
    CK(cudaStreamWaitEvent(c->s, c->ev_in, 0));
    return SSX_OK;
}
int leave(ssx_ctx *c, int rc) {
    cudaError_t e1 = cudaEventRecord(c->ev_out, c->s);
    cudaError_t e2 = cudaStreamWaitEvent(c->user, c->ev_out, 0);
    if (rc == SSX_OK && (e1 != cudaSuccess || e2 != cudaSuccess))
        return fail(c, SSX_ERR_CUDA, "stream ordering failed");
    return rc;
}
int check_sweeps(ssx_ctx *c) { return check_sweeps_quiet(c); }

int ready(ssx_ctx *c) {
    if (!c) return SSX_ERR_ARG;
    if (!c->have_model) return fail(c, SSX_ERR_ARG, "ssx_set_velocity_model not called");
    if (!c->have_geom) return fail(c, SSX_ERR_ARG, "ssx_set_geometry not called");
    return SSX_OK;
}
size_t line_bytes(ssx_ctx *c) { return (size_t)c->gd.nt * c->geom.n_line * sizeof(double); }
size_t rec_bytes(ssx_ctx *c) { return (size_t)c->gd.nt * c->geom.n_rec * sizeof(double); }

int slab_setup(ssx_ctx *c, Slab &sl, double z0, double zd, int ix0, int n) {
    const double h = c->gd.h;
    const int R = c->R;
    const int kmin = (int)std::floor(std::fmin(z0, zd) / h + 1e-6) - R;
    const int kmax = (int)std::ceil(std::fmax(z0, zd) / h - 1e-6) + R;
    TRY(grid_alloc(c, sl.g, c->gd.nx, kmax - kmin + 1, kmin, kmin * h));
    sl.z0 = z0;
    sl.zd = zd;
    sl.ix0 = ix0;
    sl.n = n;
    TRY(make_line(c, sl.g, z0, ix0, n, 1.0, &sl.plane));
    TRY(make_line(c, sl.g, zd, ix0, n, 1.0, &sl.datum));
    if (sl.tp) cudaFree(sl.tp);
    sl.tp = nullptr;
    CK(cudaMalloc(&sl.tp, 2 * (size_t)c->gd.nt * n * sizeof(double)));
    sl.tv = sl.tp + (size_t)c->gd.nt * n;
    return SSX_OK;
}

void drop_phases(ssx_ctx *c) {
    for (auto &kv : c->phases)
        if (kv.second.tabmem) cudaFree(kv.second.tabmem);
    c->phases.clear();
}

void drop_graphs(ssx_ctx *c) {
    drop_phases(c);
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    c->graph_nodes.clear();
    c->key_uses.clear();
}

// Forget tuned configurations. The captured graphs embed the configuration
// and the phase job tables, so they go too (before the tables are freed).
void reset_choices(ssx_ctx *c) {
    if (c->s) cudaStreamSynchronize(c->s);
    for (DGrid *G : {&c->full, &c->ss.g, &c->sr.g, &c->sm.g}) G->cfg[0] = G->cfg[1] = -1;
    drop_graphs(c);
}


}  // namespace

// ----------------------------------------------------------- batch solve --
// Algorithm 1 for several independent source subproblems at once (shots of
// a survey, or requests of a server), each on its own context: every PCG
// phase is one launch per time step over the union of all active shots'
// sweeps; the Krylov recurrences, scalars and stopping tests stay per shot,
// and a shot leaves the launches once it stops. Each shot's arithmetic is the
// same as in a solo solve.
struct ShotRun {
    ssx_ctx *c = nullptr;
    double alpha = 0;
    int maxit = 0;
    double rtol = 0;
    int mode = SSX_MODE_PCG;
    const double *d = nullptr;
    double *h_out = nullptr;
    double *hist = nullptr;   // host, maxit + 1 entries, may be null
    int iters = 0;
    int status = SSX_OK;
    enum { NEW, RHS, FIRST, ITER, DONE } state = NEW;
    double r0 = 0;
    std::string msg;
    bool active() const { return state != DONE; }
};

enum PhaseKind { PK_R1, PK_R2, PK_RC, PK_M1, PK_M2, PK_N1, PK_N2, PK_NC1, PK_NC2 };

void add_sweeps(ssx_ctx *c, int kind, double alpha, std::vector<Sweep> &out) {
    Slab &r = c->sr, &s = c->ss, &m = c->sm;
    const double sg = c->sgn;
    auto push = [&](Sweep w) {
        w.nt = c->gd.nt;
        out.push_back(w);
    };
    switch (kind) {
        case PK_R1: push(fwd_sweep(r.g, r.plane, nullptr, c->tr1, r.datum, r.tp, r.tv)); break;
        case PK_R2:
            push(adj_sweep(r.g, scaled(r.plane, -4.0 * sg), nullptr, c->tr2, r.datum, r.tv, r.tp));
            push(adj_sweep(c->full, c->src, c->r, nullptr, c->rec, c->tr2, nullptr, 2));
            break;
        case PK_RC: push(adj_sweep(c->full, c->src, c->r, nullptr, c->rec, c->tr1, nullptr)); break;
        case PK_M1: push(fwd_sweep(s.g, s.plane, nullptr, c->tl1, s.datum, s.tp, s.tv)); break;
        case PK_M2:
            push(adj_sweep(s.g, scaled(s.plane, -4.0 * sg), nullptr, c->tl2, s.datum, s.tv, s.tp));
            break;
        case PK_N1:
            push(fwd_sweep(c->full, c->src, c->p, nullptr, c->rec, c->tr1, nullptr));
            push(fwd_sweep(r.g, r.plane, nullptr, c->tr1, r.datum, r.tp, r.tv, 1));
            if (alpha != 0.0) push(fwd_sweep(m.g, m.plane, c->tl1, nullptr, m.datum, m.tp, m.tv));
            break;
        case PK_N2:
            push(adj_sweep(r.g, scaled(r.plane, -4.0 * sg), nullptr, c->tr2, r.datum, r.tv, r.tp));
            push(adj_sweep(c->full, c->src, c->q, nullptr, c->rec, c->tr2, nullptr, 2));
            if (alpha != 0.0)
                push(adj_sweep(m.g, scaled(m.plane, -1.0 * sg), c->tl2, nullptr, m.datum, m.tv, m.tp));
            break;
        case PK_NC1: push(fwd_sweep(c->full, c->src, c->p, nullptr, c->rec, c->tr1, nullptr)); break;
        case PK_NC2: push(adj_sweep(c->full, c->src, c->q, nullptr, c->rec, c->tr1, nullptr)); break;
    }
}

// One round of the solve engine for a set of shots (each at its own stage of
// Algorithm 1). A shot's stages: NEW (set-up of r_0 = S^* d: the two R
// phases), FIRST (g_0 = M^{-1} r_0, p_0 = g_0, q_0 = N p_0) and ITER (one
// update h += alpha p, r -= alpha q with its stopping test, then
// g = M^{-1} r, p = g + beta p, q = N p). Every round runs the same four
// phases; each shot contributes the sweeps of its stage (the R phases of new
// shots share launches with the M phases of the others), so shots can join at
// any round. The per-shot arithmetic is the same whatever else shares the
// launches.
int engine_round(ssx_ctx *L, std::vector<ShotRun *> &shots) {
    ssx_ctx *c = L;   // for CK/TRY error reporting
    cudaStream_t s = L->s;
    auto nl = [](ShotRun &sh) { return (size_t)sh.c->gd.nt * sh.c->geom.n_line; };
    auto stop = [&](ShotRun &sh, int status, const std::string &msg) {
        sh.status = status;
        sh.msg = msg;
        sh.state = ShotRun::DONE;
    };
    // --- update step of iterating shots and the residual norms -------------
    bool any_read = false;
    for (ShotRun *p : shots) {
        ShotRun &sh = *p;
        if (sh.state == ShotRun::ITER) {
            double *sc = sh.c->sc;
            CK(launch_dot(sh.c->p, sh.c->q, nl(sh), sh.c->partials, sc + SC_PQ, s));
            if (sh.c->hook != SSX_HOOK_NONE && sh.c->hook_k == sh.iters) {
                // test hook: <p_k, q_k> replaced (0, or a NaN pattern) before alpha_k
                CK(cudaMemsetAsync(sc + SC_PQ, sh.c->hook == SSX_HOOK_BREAKDOWN ? 0 : 0xff,
                                   sizeof(double), s));
                sh.c->hook = SSX_HOOK_NONE;
            }
            CK(launch_pcg_alpha(sc, s));
            CK(launch_pcg_update(sh.c->h, sh.c->r, sh.c->p, sh.c->q, nl(sh), sc, sh.c->partials, s));
            L->st.kernel_launches += 5;
        }
        if (sh.state == ShotRun::ITER || sh.state == ShotRun::RHS) {
            CK(cudaMemcpyAsync(sh.c->sc_host, sh.c->sc, SC_COUNT * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
            any_read = true;
        }
    }
    if (any_read) CK(cudaStreamSynchronize(s));
    for (ShotRun *p : shots) {
        ShotRun &sh = *p;
        const double *h = sh.c->sc_host;
        if (sh.state == ShotRun::RHS) {   // r_0 known
            sh.r0 = std::sqrt(h[SC_RR]);
            if (sh.hist) sh.hist[0] = sh.r0;
            if (!std::isfinite(sh.r0)) stop(sh, SSX_ERR_NONFINITE, "non-finite initial residual");
            else if (sh.r0 == 0.0) stop(sh, SSX_OK, "");
            else if (sh.maxit == 0) stop(sh, SSX_ERR_NOT_CONVERGED, "maxit reached above rtol");
            else sh.state = ShotRun::FIRST;
        } else if (sh.state == ShotRun::ITER) {
            const int k = sh.iters;
            if (h[SC_FLAG] != 0.0) {
                if (!std::isfinite(h[SC_PQ]) || !std::isfinite(h[SC_GR])) {
                    stop(sh, SSX_ERR_NONFINITE, "non-finite Krylov scalar");
                } else {
                    char b[160];
                    snprintf(b, sizeof b, "PCG breakdown at k=%d: <p,q>=%.6e <g,r>=%.6e", k,
                             h[SC_PQ], h[SC_GR]);
                    stop(sh, SSX_ERR_BREAKDOWN, b);
                }
                continue;
            }
            const double rn = std::sqrt(h[SC_RR]);
            sh.iters = k + 1;
            if (sh.hist) sh.hist[k + 1] = rn;
            if (!std::isfinite(rn)) stop(sh, SSX_ERR_NONFINITE, "non-finite residual");
            else if (rn <= sh.rtol * sh.r0) stop(sh, SSX_OK, "");
            else if (k == sh.maxit - 1) stop(sh, SSX_ERR_NOT_CONVERGED, "maxit reached above rtol");
        }
    }
    // --- the four phases ----------------------------------------------------
    auto want_M = [](const ShotRun &sh) {
        return sh.state == ShotRun::FIRST || sh.state == ShotRun::ITER;
    };
    auto phase = [&](const char *name, const std::function<void(ShotRun &, std::vector<Sweep> &)> &f) -> int {
        std::vector<Sweep> sw;
        for (ShotRun *p : shots) f(*p, sw);
        return sw.empty() ? SSX_OK : run_phase(L, name, sw);
    };
    // new shots: d -> tr1, h = 0
    for (ShotRun *p : shots) {
        ShotRun &sh = *p;
        if (sh.state != ShotRun::NEW) continue;
        if (sh.mode == SSX_MODE_PCG) TRY(set_D(sh.c, sh.alpha));
        CK(cudaMemcpyAsync(sh.c->tr1, sh.d, rec_bytes(sh.c), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(sh.c->h, 0, line_bytes(sh.c), s));
    }
    // M^{-1} input D r (PCG)
    for (ShotRun *p : shots) {
        ShotRun &sh = *p;
        if (want_M(sh) && sh.mode == SSX_MODE_PCG) {
            CK(launch_colscale(sh.c->tl1, sh.c->r, sh.c->D, sh.c->gd.nt, sh.c->geom.n_line, s));
            L->st.kernel_launches += 1;
        }
    }
    TRY(phase("e1", [&](ShotRun &sh, std::vector<Sweep> &sw) {
        if (sh.state == ShotRun::NEW) add_sweeps(sh.c, sh.mode == SSX_MODE_PCG ? PK_R1 : PK_RC, sh.alpha, sw);
        else if (want_M(sh) && sh.mode == SSX_MODE_PCG) add_sweeps(sh.c, PK_M1, sh.alpha, sw);
    }));
    TRY(phase("e2", [&](ShotRun &sh, std::vector<Sweep> &sw) {
        if (sh.state == ShotRun::NEW && sh.mode == SSX_MODE_PCG) add_sweeps(sh.c, PK_R2, sh.alpha, sw);
        else if (want_M(sh) && sh.mode == SSX_MODE_PCG) add_sweeps(sh.c, PK_M2, sh.alpha, sw);
    }));
    for (ShotRun *p : shots) {
        ShotRun &sh = *p;
        if (sh.state == ShotRun::NEW) {   // ||r_0||^2, read next round
            CK(launch_dot(sh.c->r, sh.c->r, nl(sh), sh.c->partials, sh.c->sc + SC_RR, s));
            L->st.kernel_launches += 2;
            continue;
        }
        if (!want_M(sh)) continue;
        if (sh.mode == SSX_MODE_PCG) {
            CK(launch_colscale(sh.c->g, sh.c->tl2, sh.c->D, sh.c->gd.nt, sh.c->geom.n_line, s));
            L->st.kernel_launches += 1;
        } else {
            CK(cudaMemcpyAsync(sh.c->g, sh.c->r, nl(sh) * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        if (sh.state == ShotRun::FIRST) {   // p_0 = g_0, <g_0, r_0>
            CK(cudaMemcpyAsync(sh.c->p, sh.c->g, line_bytes(sh.c), cudaMemcpyDeviceToDevice, s));
            CK(launch_dot(sh.c->g, sh.c->r, nl(sh), sh.c->partials, sh.c->sc + SC_GR, s));
            L->st.kernel_launches += 2;
        } else {                            // beta, p = g + beta p
            double *sc = sh.c->sc;
            CK(launch_dot(sh.c->g, sh.c->r, nl(sh), sh.c->partials, sc + SC_GRNEW, s));
            CK(launch_pcg_beta(sc, s));
            CK(launch_xpby(sh.c->p, sh.c->g, nl(sh), sc, s));
            L->st.kernel_launches += 4;
        }
        if (sh.mode == SSX_MODE_PCG && sh.alpha != 0.0) {   // A p for W~_m
            CK(launch_colscale(sh.c->tl1, sh.c->p, sh.c->dist, sh.c->gd.nt, sh.c->geom.n_line, s));
            L->st.kernel_launches += 1;
        }
    }
    TRY(phase("e3", [&](ShotRun &sh, std::vector<Sweep> &sw) {
        if (want_M(sh)) add_sweeps(sh.c, sh.mode == SSX_MODE_PCG ? PK_N1 : PK_NC1, sh.alpha, sw);
    }));
    TRY(phase("e4", [&](ShotRun &sh, std::vector<Sweep> &sw) {
        if (want_M(sh)) add_sweeps(sh.c, sh.mode == SSX_MODE_PCG ? PK_N2 : PK_NC2, sh.alpha, sw);
    }));
    for (ShotRun *p : shots) {
        ShotRun &sh = *p;
        if (want_M(sh) && sh.alpha != 0.0) {
            if (sh.mode == SSX_MODE_PCG)
                CK(launch_colscale_add(sh.c->q, sh.c->tl2, sh.c->dist, sh.alpha, sh.c->gd.nt,
                                       sh.c->geom.n_line, s));
            else
                CK(launch_colscale_add(sh.c->q, sh.c->p, sh.c->dist2, sh.alpha, sh.c->gd.nt,
                                       sh.c->geom.n_line, s));
            L->st.kernel_launches += 1;
        }
        if (sh.state == ShotRun::NEW) sh.state = ShotRun::RHS;
        else if (sh.state == ShotRun::FIRST) sh.state = ShotRun::ITER;
    }
    return SSX_OK;
}

// finished shots: the last iterate to the caller's buffer
int engine_retire(ssx_ctx *L, ShotRun &sh) {
    ssx_ctx *c = L;
    if (sh.h_out)
        CK(cudaMemcpyAsync(sh.h_out, sh.c->h, line_bytes(sh.c), cudaMemcpyDeviceToDevice, L->s));
    if (sh.status != SSX_OK) sh.c->err = sh.msg;
    return SSX_OK;
}

int solve_batch(std::vector<ShotRun> &shots) {
    ssx_ctx *L = shots[0].c;
    std::vector<ShotRun *> act;
    for (auto &sh : shots) act.push_back(&sh);
    while (true) {
        bool any = false;
        for (auto &sh : shots) any = any || sh.active();
        if (!any) break;
        TRY(engine_round(L, act));
    }
    for (auto &sh : shots) TRY(engine_retire(L, sh));
    return SSX_OK;
}

// ---------------------------------------------------------------- server --
// Continuous batching of source-subproblem solves: requests queue up, are
// admitted while their estimated device memory fits the budget, join the
// engine at the next round (sharing every launch with the solves already
// running), and leave when they stop, freeing their memory for the queue.
// Device memory of a request's grids (the full grid and its three slabs:
// kappa, two ping-pong field triples and C_p each), which its sweeps step
// through every phase: the request's working set.
static size_t field_bytes(const ssx_grid_desc &g, const ssx_geom_desc &m) {
    const int nsp = g.n_sponge;
    auto grid_bytes = [&](int nx, int nz) {
        const FieldLayout L = field_layout(nx + 2 * nsp, nz + 2 * nsp);
        return 8 * L.elems() * sizeof(float) + (size_t)4096 * 4;
    };
    const int slab_rows = (int)std::ceil(m.dz_datum / g.h) + 3 + g.space_order;
    return grid_bytes(g.nx, g.nz) + 3 * grid_bytes(g.nx, slab_rows);
}

// A request's device memory: its grids, gathers and model copy.
static size_t estimate_bytes(const ssx_grid_desc &g, const ssx_geom_desc &m) {
    const size_t nl = (size_t)g.nt * m.n_line, nr = (size_t)g.nt * m.n_rec;
    return field_bytes(g, m) + (7 * nl + 2 * nr + 4 * nl + 2 * nr) * 8 + (size_t)g.nx * g.nz * 4 +
           ((size_t)1 << 20);
}

struct ssx_server {
    struct Req {
        int id = 0;
        ssx_grid_desc g{};
        ssx_geom_desc m{};
        const float *v = nullptr;
        double rho = 1.0;
        ShotRun run;
        ssx_ctx *c = nullptr;
        size_t bytes = 0, ws = 0;   // device memory, working set (field_bytes)
        double t_submit = 0, t_admit = 0, t_done = 0;
        bool done = false;
    };
    ssx_ctx *lead = nullptr;       // owns the stream, the phase launches and their statistics
    size_t budget = 0, used = 0;
    // admission also keeps the active requests' working sets within this many
    // bytes (the L2 cache by default; 0: no limit), so that a batch's fields
    // stay cache-resident between time steps
    size_t cache_budget = 0, used_ws = 0;
    int order = 8;
    int next_id = 1;
    std::deque<Req *> queue;
    std::vector<Req *> active;
    std::unordered_map<int, Req *> all;
    std::string err;
    long long rounds = 0, request_rounds = 0;   // engine rounds run, and requests in them
};

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int server_admit(ssx_server *sv) {
    while (!sv->queue.empty()) {
        ssx_server::Req *q = sv->queue.front();
        // first in, first out: the head waits until it fits (or runs alone)
        if (!sv->active.empty() &&
            (sv->used + q->bytes > sv->budget ||
             (sv->cache_budget && sv->used_ws + q->ws > sv->cache_budget)))
            break;
        sv->queue.pop_front();
        ssx_ctx *c = nullptr;
        int rc = ssx_create(&c, &q->g, sv->lead->user);
        if (rc == SSX_OK) rc = ssx_set_velocity_model(c, q->v, q->rho);
        if (rc == SSX_OK) rc = ssx_set_geometry(c, &q->m);
        if (rc != SSX_OK) {
            q->run.status = rc;
            q->run.msg = c ? c->err : "context creation failed";
            q->done = true;
            q->t_done = now_ms();
            if (c) ssx_destroy(c);
            continue;
        }
        q->c = c;
        q->run.c = c;
        q->t_admit = now_ms();
        sv->used += q->bytes;
        sv->used_ws += q->ws;
        sv->active.push_back(q);
    }
    return SSX_OK;
}

}  // namespace

// ================================================================ C ABI ==
extern "C" {

const char *ssx_version(void) { return "ssx 0.1 (sm_103a)"; }

const char *ssx_last_error(const ssx_ctx *c) { return c ? c->err.c_str() : "null context"; }

int ssx_create(ssx_ctx **out, const ssx_grid_desc *gd, void *stream) {
    if (!out || !gd) return SSX_ERR_ARG;
    *out = nullptr;
    if (gd->nx < 8 || gd->nz < 8 || gd->nt < 1 || !(gd->h > 0) || !(gd->dt > 0) ||
        gd->n_sponge < 0 || gd->space_order < 2 || gd->space_order > 8 || gd->space_order % 2)
        return SSX_ERR_ARG;
    if ((long long)(gd->nx + 2 * gd->n_sponge) * (gd->nz + 2 * gd->n_sponge) > (1LL << 28))
        return SSX_ERR_ARG;
    ssx_ctx *c = new ssx_ctx();
    c->gd = *gd;
    c->R = gd->space_order / 2;
    c->user = (cudaStream_t)stream;
    int rc = SSX_OK;
    auto init = [&]() -> int {
        for (auto &row : c->cap) row[0] = row[1] = -1;
        for (int &v : c->tma_cap) v = -1;
        for (int &v : c->march_cap) v = -1;
        // SSX_GRAPHS=0: launch every step directly instead of replaying CUDA
        // graphs (profilers treat each graph replay as a rebuild)
        if (const char *e = std::getenv("SSX_GRAPHS")) c->use_graphs = std::strcmp(e, "0") != 0;
        if (const char *e = std::getenv("SSX_LOG_TUNING")) c->log_tuning = std::strcmp(e, "1") == 0;
        CK(prepare_kernels());
        CK(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
        CK(cudaMalloc(&c->vel, (size_t)gd->nx * gd->nz * sizeof(float)));
        CK(cudaMalloc(&c->vmax_dev, sizeof(float)));
        CK(cudaMalloc(&c->sc, SC_COUNT * sizeof(double)));
        CK(cudaMalloc(&c->partials, kDotBlocks * sizeof(double)));
        CK(cudaMallocHost(&c->sc_host, (SC_COUNT + 1) * sizeof(double)));
        CK(cudaMalloc(&c->d_err, sizeof(int)));
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->s));
        TRY(grid_alloc(c, c->full, gd->nx, gd->nz, 0, 0.0));
        CK(cudaStreamSynchronize(c->s));
        return SSX_OK;
    };
    rc = init();
    if (rc != SSX_OK) {
        ssx_destroy(c);
        return rc;
    }
    *out = c;
    return SSX_OK;
}

int ssx_destroy(ssx_ctx *c) {
    if (!c) return SSX_ERR_ARG;
    if (c->s) cudaStreamSynchronize(c->s);
    drop_graphs(c);
    for (auto &e : c->evs) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    grid_free(c->full);
    grid_free(c->ss.g);
    grid_free(c->sm.g);
    if (c->sm.tp) cudaFree(c->sm.tp);
    grid_free(c->sr.g);
    if (c->ss.tp) cudaFree(c->ss.tp);
    if (c->sr.tp) cudaFree(c->sr.tp);
    if (c->gbuf) cudaFree(c->gbuf);
    if (c->vel) cudaFree(c->vel);
    if (c->vmax_dev) cudaFree(c->vmax_dev);
    if (c->sc) cudaFree(c->sc);
    if (c->partials) cudaFree(c->partials);
    if (c->sc_host) cudaFreeHost(c->sc_host);
    if (c->d_err) cudaFree(c->d_err);
    if (c->gw) cudaFree(c->gw);
    if (c->gwd) cudaFree(c->gwd);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->s) cudaStreamDestroy(c->s);
    delete c;
    return SSX_OK;
}

int ssx_set_velocity_model(ssx_ctx *c, const float *v_dev, double rho) {
    if (!c || !v_dev || !(rho > 0)) return c ? fail(c, SSX_ERR_ARG, "bad model arguments") : SSX_ERR_ARG;
    TRY(enter(c));
    auto body = [&]() -> int {
        const size_t n = (size_t)c->gd.nx * c->gd.nz;
        CK(cudaMemcpyAsync(c->vel, v_dev, n * sizeof(float), cudaMemcpyDeviceToDevice, c->s));
        CK(launch_vmax(c->vel, (int)n, c->vmax_dev, c->s));
        float vm = 0.f;
        CK(cudaMemcpyAsync(&vm, c->vmax_dev, sizeof(float), cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
        if (!(vm > 0) || !std::isfinite(vm)) return fail(c, SSX_ERR_ARG, "velocity must be positive");
        const double cfl = vm * c->gd.dt / c->gd.h * std::sqrt(2.0) * kWeightsAbsSum[c->R];
        if (!(cfl < 1.0)) {
            char b[128];
            snprintf(b, sizeof b, "CFL violated: v_max dt/h sqrt(2) sum|c| = %.4f >= 1", cfl);
            return fail(c, SSX_ERR_CFL, b);
        }
        c->v_max = vm;
        c->rho = rho;
        drop_graphs(c);   // captured sweeps and job tables hold the old coefficients
        TRY(grid_fill(c, c->full));
        if (c->have_geom) {
            TRY(grid_fill(c, c->ss.g));
            TRY(grid_fill(c, c->sr.g));
            TRY(grid_fill(c, c->sm.g));
        }
        c->have_model = true;
        return SSX_OK;
    };
    return leave(c, body());
}

int ssx_set_geometry(ssx_ctx *c, const ssx_geom_desc *gm) {
    if (!c || !gm) return c ? fail(c, SSX_ERR_ARG, "null geometry") : SSX_ERR_ARG;
    const double h = c->gd.h;
    const double zmax = (c->gd.nz - 1) * h;
    if (gm->z_s < -1e-9 || gm->z_s > zmax + 1e-9 || gm->z_r < -1e-9 || gm->z_r > zmax + 1e-9)
        return fail(c, SSX_ERR_ARG, "z_s and z_r must lie in the physical model");
    if (std::fabs(gm->z_s - gm->z_r) < h) return fail(c, SSX_ERR_ARG, "z_s and z_r must differ by >= h");
    if (!(gm->dz_datum >= h)) return fail(c, SSX_ERR_ARG, "dz_datum must be >= h");
    TRY(enter(c));
    auto body = [&]() -> int {
        CK(cudaStreamSynchronize(c->s));
        drop_graphs(c);
        c->have_geom = false;
        TRY(make_line(c, c->full, gm->z_s, gm->ix_line0, gm->n_line, 1.0, &c->src));
        TRY(make_line(c, c->full, gm->z_r, gm->ix_rec0, gm->n_rec, 1.0, &c->rec));
        c->geom = *gm;
        const double dir = gm->z_r > gm->z_s ? 1.0 : -1.0;
        c->sgn = -dir;
        TRY(slab_setup(c, c->ss, gm->z_s, gm->z_s + dir * gm->dz_datum, gm->ix_line0, gm->n_line));
        TRY(slab_setup(c, c->sr, gm->z_r, gm->z_r + dir * gm->dz_datum, gm->ix_rec0, gm->n_rec));
        TRY(slab_setup(c, c->sm, gm->z_s, gm->z_s + dir * gm->dz_datum, gm->ix_line0, gm->n_line));
        if (c->gbuf) cudaFree(c->gbuf);
        c->gbuf = nullptr;
        const size_t nl = (size_t)c->gd.nt * gm->n_line, nr = (size_t)c->gd.nt * gm->n_rec;
        CK(cudaMalloc(&c->gbuf, (7 * nl + 2 * nr + 3 * (size_t)gm->n_line) * sizeof(double)));
        double *b = c->gbuf;
        c->h = b; b += nl;
        c->r = b; b += nl;
        c->g = b; b += nl;
        c->p = b; b += nl;
        c->q = b; b += nl;
        c->tl1 = b; b += nl;
        c->tl2 = b; b += nl;
        c->tr1 = b; b += nr;
        c->tr2 = b; b += nr;
        c->dist = b; b += gm->n_line;
        c->dist2 = b; b += gm->n_line;
        c->D = b;
        c->D_alpha = -1.0;
        std::vector<double> dd(2 * (size_t)gm->n_line);
        for (int j = 0; j < gm->n_line; j++) {
            const double x = (gm->ix_line0 + j) * h - gm->x_s;
            dd[j] = std::fabs(x);
            dd[gm->n_line + j] = x * x;
        }
        CK(cudaMemcpyAsync(c->dist, dd.data(), dd.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
        if (c->have_model) {
            TRY(grid_fill(c, c->ss.g));
            TRY(grid_fill(c, c->sr.g));
            TRY(grid_fill(c, c->sm.g));
        }
        CK(cudaStreamSynchronize(c->s));
        c->have_geom = true;
        return SSX_OK;
    };
    return leave(c, body());
}

int ssx_forward(ssx_ctx *c, const double *h_dev, double *d_dev) {
    TRY(ready(c));
    if (!h_dev || !d_dev) return fail(c, SSX_ERR_ARG, "null gather");
    TRY(enter(c));
    auto body = [&]() -> int {
        CK(cudaMemcpyAsync(c->tl1, h_dev, line_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        TRY(op_S(c, c->tl1, c->tr1));
        CK(cudaMemcpyAsync(d_dev, c->tr1, rec_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        return check_sweeps(c);
    };
    return leave(c, body());
}

// ------------------------------------------------------- velocity gradient --
// dPhi/dv of Phi = ||S[v] h - d||^2 + alpha ||A h||^2 at fixed h (the reduced
// objective's gradient when h solves eqn:esis), by the discrete adjoint state
// method with uniform checkpoints:
//   1. forward sweep of S h from rest, saving the state (p, v_x, v_z) before
//      every K-th step, and the traces y;
//   2. ybar = 2 (y - d), Phi from the two norms;
//   3. the transposed sweep driven by ybar, run backwards segment by segment:
//      each segment's forward pressures p^{n0} .. p^{n1} are recomputed from
//      its checkpoint (same kernels, so bit for bit the first sweep's), then
//      its reverse steps run, each preceded by the accumulation of
//      pbar^{n+1} (p^{n+1} - A_p p^n) / kappa~ into the FP64 gradient;
//   4. the padded-grid sum is folded onto the physical model.
// Phi of the last gradient: ||y - d||^2 = |ybar|^2 / 4 and ||A h||^2, the two
// scalars after the gradient's trace and penalty buffers (synchronises)
static int last_objective(ssx_ctx *c, double *objective) {
    if (!c->have_grad) return fail(c, SSX_ERR_ARG, "no velocity gradient computed yet");
    const int nt = c->gd.nt;
    const size_t NP = (size_t)c->full.L.NX * c->full.L.NZ;
    const double *sc = c->gwd + NP + 2 * (size_t)nt * c->geom.n_rec + (size_t)nt * c->geom.n_line;
    CK(cudaMemcpyAsync(c->sc_host, sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    *objective = 0.25 * c->sc_host[0] + c->grad_alpha * c->sc_host[1];
    return SSX_OK;
}

static int velocity_gradient(ssx_ctx *c, const double *h, const double *d, double alpha, int K,
                             double *grad, double *objective) {
    DGrid &G = c->full;
    const int nt = c->gd.nt, R = c->R;
    const int nrec = c->geom.n_rec, nl = c->geom.n_line;
    TRY(select_config(c, G, false));
    TRY(select_config(c, G, true));
    const int cf = G.cfg[0], ca = G.cfg[1];   // step launches (never the persistent form)
    const size_t E = G.L.elems(), org = G.L.origin();
    const int ncp = (nt + K - 1) / K, seg = std::min(K, nt);
    // floats: checkpoints [ncp][3][E] | p slots [seg+1][E] | v_x, v_z [2][2][E] | adjoint [2][3][E]
    const size_t nf = ((size_t)ncp * 3 + (size_t)seg + 1 + 4 + 6) * E;
    // doubles: accumulator [NZ][NX] | y, ybar [nt][nrec] | A h [nt][nl] | 2 scalars
    const size_t NP = (size_t)G.L.NX * G.L.NZ;
    const size_t nd = NP + 2 * (size_t)nt * nrec + (size_t)nt * nl + 2;
    if (c->gw_floats < nf) {
        if (c->gw) CK(cudaFree(c->gw));
        c->gw = nullptr;
        c->gw_floats = 0;
        CK(cudaMalloc(&c->gw, nf * sizeof(float)));
        c->gw_floats = nf;
    }
    if (c->gw_doubles < nd) {
        if (c->gwd) CK(cudaFree(c->gwd));
        c->gwd = nullptr;
        c->gw_doubles = 0;
        CK(cudaMalloc(&c->gwd, nd * sizeof(double)));
        c->gw_doubles = nd;
    }
    float *cp = c->gw;                                    // checkpoints
    float *slot = cp + (size_t)ncp * 3 * E;               // recomputed p^n
    float *vbuf = slot + (size_t)(seg + 1) * E;           // [vx0 vz0 vx1 vz1]
    float *abuf = vbuf + 4 * E;                           // adjoint [p vx vz] x 2
    double *gacc = c->gwd, *y = gacc + NP, *ybar = y + (size_t)nt * nrec;
    double *ah = ybar + (size_t)nt * nrec, *sc = ah + (size_t)nt * nl;
    // the launches, captured once per set of buffers into a CUDA graph (an
    // outer loop recomputes gradients on the same buffers) and replayed
    auto enqueue = [&](cudaStream_t s) -> int {
    // every field array starts from zeros: the aprons are never written
    CK(cudaMemsetAsync(slot, 0, (size_t)(seg + 1 + 4 + 6) * E * sizeof(float), s));
    CK(cudaMemsetAsync(gacc, 0, NP * sizeof(double), s));
    CK(cudaMemsetAsync(y, 0, (size_t)nt * nrec * sizeof(double), s));
    CK(cudaMemsetAsync(G.mem + E, 0, 3 * E * sizeof(float), s));
    auto F = [&](float *base) { return base + org; };   // origin-offset field pointer

    // 1. forward sweep with checkpoints and traces
    FwdArgs a{};
    a.g = G.args;
    a.src = c->src;
    a.hsrc = h;
    a.rec = c->rec;
    a.outp = y;
    for (int n = 0; n < nt; n++) {
        const int bi = n & 1, bo = bi ^ 1;
        if (n % K == 0)
            for (int f = 0; f < 3; f++)
                CK(cudaMemcpyAsync(cp + ((size_t)(n / K) * 3 + f) * E, G.f[bi][f] - org,
                                   E * sizeof(float), cudaMemcpyDeviceToDevice, s));
        a.p_in = G.f[bi][0];
        a.vx_in = G.f[bi][1];
        a.vz_in = G.f[bi][2];
        a.p_out = G.f[bo][0];
        a.vx_out = G.f[bo][1];
        a.vz_out = G.f[bo][2];
        a.n = n;
        CK(launch_fwd_step(a, R, cf, s, true));
    }
    // 2. residual and objective
    CK(launch_residual2(ybar, y, d, (size_t)nt * nrec, s));
    CK(launch_dot(ybar, ybar, (size_t)nt * nrec, c->partials, sc, s));
    CK(launch_colscale(ah, h, c->dist, nt, nl, s));
    CK(launch_dot(ah, ah, (size_t)nt * nl, c->partials, sc + 1, s));

    // 3. transposed sweep of ybar, segments in reverse, with recompute
    AdjArgs b{};
    b.g = G.args;
    b.src = c->src;
    b.rec = c->rec;
    b.yp = ybar;
    float *A[2][3];
    for (int q = 0; q < 2; q++)
        for (int f = 0; f < 3; f++) A[q][f] = F(abuf + (size_t)(3 * q + f) * E);
    b.p_in = A[0][0];
    b.vx_in = A[0][1];
    b.vz_in = A[0][2];
    CK(launch_adj_init(b, nt, s));
    FwdArgs r{};
    r.g = G.args;
    r.src = c->src;
    r.hsrc = h;
    r.rec = c->rec;
    r.rec.n = 0;   // recompute: no sampling
    for (int k = ncp - 1; k >= 0; k--) {
        const int n0 = k * K, n1 = std::min(nt, n0 + K);
        CK(cudaMemcpyAsync(slot, cp + (size_t)k * 3 * E, E * sizeof(float), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(vbuf, cp + ((size_t)k * 3 + 1) * E, 2 * E * sizeof(float),
                           cudaMemcpyDeviceToDevice, s));
        for (int n = n0; n < n1; n++) {
            const int vi = (n - n0) & 1, vo = vi ^ 1;
            r.p_in = F(slot + (size_t)(n - n0) * E);
            r.p_out = F(slot + (size_t)(n - n0 + 1) * E);
            r.vx_in = F(vbuf + (size_t)(2 * vi) * E);
            r.vz_in = F(vbuf + (size_t)(2 * vi + 1) * E);
            r.vx_out = F(vbuf + (size_t)(2 * vo) * E);
            r.vz_out = F(vbuf + (size_t)(2 * vo + 1) * E);
            r.n = n;
            CK(launch_fwd_step(r, R, cf, s, true));
        }
        for (int n = n1 - 1; n >= n0; n--) {
            const int t = nt - 1 - n, bi = t & 1, bo = bi ^ 1;
            CK(launch_grad_accum(gacc, A[bi][0], F(slot + (size_t)(n + 1 - n0) * E),
                                 F(slot + (size_t)(n - n0) * E), G.args, s));
            b.p_in = A[bi][0];
            b.vx_in = A[bi][1];
            b.vz_in = A[bi][2];
            b.p_out = A[bo][0];
            b.vx_out = A[bo][1];
            b.vz_out = A[bo][2];
            b.n = n;
            CK(launch_adj_step(b, R, ca, s, true));
        }
    }
    // 4. onto the physical model: dPhi/dv = 2 rho v (dt/h) sum dPhi/dkappa~
    CK(launch_grad_fold(grad, gacc, c->vel, G.args.kap, G.L.pitch, c->gd.nx, c->gd.nz, c->gd.n_sponge, G.L.NX,
                        2.0 * c->rho * c->gd.dt / c->gd.h, s));
    return SSX_OK;
    };
    char key[256];
    snprintf(key, sizeof key, "grad:%p:%p:%p:%p:%p:%d:%d:%d:%d", (const void *)h, (const void *)d,
             (void *)grad, (void *)c->gw, (void *)c->gwd, K, nt, cf, ca);
    TRY(run_cached(c, key, 4LL * nt + 6, 3LL * nt, 3.0 * G.L.NX * G.L.NZ * nt, enqueue));
    c->grad_alpha = alpha;
    c->have_grad = true;
    if (objective) TRY(last_objective(c, objective));
    return SSX_OK;
}

int ssx_velocity_gradient(ssx_ctx *c, const double *h_dev, const double *d_dev, double alpha,
                          int checkpoint_every, double *grad_dev, double *objective) {
    TRY(ready(c));
    if (!h_dev || !d_dev || !grad_dev) return fail(c, SSX_ERR_ARG, "null argument");
    if (checkpoint_every < 1) return fail(c, SSX_ERR_ARG, "checkpoint_every must be >= 1");
    if (!(alpha >= 0.0)) return fail(c, SSX_ERR_ARG, "alpha must be >= 0");
    TRY(enter(c));
    // step kernels only (no bounded waits, so no timeout flag to read): without
    // objective_host the call returns as soon as its work is queued
    const int rc = velocity_gradient(c, h_dev, d_dev, alpha, checkpoint_every, grad_dev, objective);
    return leave(c, rc);
}

int ssx_last_objective(ssx_ctx *c, double *objective_host) {
    if (!c) return SSX_ERR_ARG;
    if (!objective_host) return fail(c, SSX_ERR_ARG, "null argument");
    return last_objective(c, objective_host);
}

int ssx_adjoint(ssx_ctx *c, const double *d_dev, double *h_dev) {
    TRY(ready(c));
    if (!h_dev || !d_dev) return fail(c, SSX_ERR_ARG, "null gather");
    TRY(enter(c));
    auto body = [&]() -> int {
        CK(cudaMemcpyAsync(c->tr2, d_dev, rec_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        TRY(op_ST(c, c->tr2, c->tl2));
        CK(cudaMemcpyAsync(h_dev, c->tl2, line_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        return check_sweeps(c);
    };
    return leave(c, body());
}

int ssx_weight_apply(ssx_ctx *c, int which, const double *in, double *out) {
    TRY(ready(c));
    if (!in || !out) return fail(c, SSX_ERR_ARG, "null gather");
    if (which != SSX_W_D && which != SSX_W_M && which != SSX_W_M_INV)
        return fail(c, SSX_ERR_ARG, "unknown weight operator");
    TRY(enter(c));
    auto body = [&]() -> int {
        const bool rec = which == SSX_W_D;
        double *bi = rec ? c->tr1 : c->tl1;
        double *bo = rec ? c->tr2 : c->tl2;
        const size_t bytes = rec ? rec_bytes(c) : line_bytes(c);
        CK(cudaMemcpyAsync(bi, in, bytes, cudaMemcpyDeviceToDevice, c->s));
        TRY(op_W(c, which, bi, bo));
        CK(cudaMemcpyAsync(out, bo, bytes, cudaMemcpyDeviceToDevice, c->s));
        return check_sweeps(c);
    };
    return leave(c, body());
}

int ssx_lambda_apply(ssx_ctx *c, int transpose, const double *in, double *out) {
    TRY(ready(c));
    if (!in || !out) return fail(c, SSX_ERR_ARG, "null gather");
    TRY(enter(c));
    auto body = [&]() -> int {
        CK(cudaMemcpyAsync(c->tl1, in, line_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        TRY(op_lambda(c, transpose != 0, c->tl1, c->tl2));
        CK(cudaMemcpyAsync(out, c->tl2, line_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        return check_sweeps(c);
    };
    return leave(c, body());
}

int ssx_time_reversal_inverse(ssx_ctx *c, const double *d_dev, double *h_dev) {
    TRY(ready(c));
    if (!d_dev || !h_dev) return fail(c, SSX_ERR_ARG, "null gather");
    TRY(enter(c));
    auto body = [&]() -> int {
        CK(cudaMemcpyAsync(c->tr1, d_dev, rec_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        TRY(op_trinv(c, c->tr1, c->tl2));
        CK(cudaMemcpyAsync(h_dev, c->tl2, line_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        return check_sweeps(c);
    };
    return leave(c, body());
}

int ssx_precond_apply(ssx_ctx *c, double alpha, const double *r, double *g) {
    TRY(ready(c));
    if (!r || !g || !(alpha >= 0)) return fail(c, SSX_ERR_ARG, "bad arguments");
    TRY(enter(c));
    auto body = [&]() -> int {
        CK(cudaMemcpyAsync(c->r, r, line_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        TRY(op_Minv(c, SSX_MODE_PCG, alpha, c->r, c->g));
        CK(cudaMemcpyAsync(g, c->g, line_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        return check_sweeps(c);
    };
    return leave(c, body());
}

int ssx_normal_apply(ssx_ctx *c, int mode, double alpha, const double *p, double *q) {
    TRY(ready(c));
    if (!p || !q || !(alpha >= 0) || (mode != SSX_MODE_PCG && mode != SSX_MODE_CG))
        return fail(c, SSX_ERR_ARG, "bad arguments");
    TRY(enter(c));
    auto body = [&]() -> int {
        CK(cudaMemcpyAsync(c->p, p, line_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        TRY(op_N(c, mode, alpha, c->p, c->q));
        CK(cudaMemcpyAsync(q, c->q, line_bytes(c), cudaMemcpyDeviceToDevice, c->s));
        return check_sweeps(c);
    };
    return leave(c, body());
}

int ssx_solve_source_subproblem(ssx_ctx *c, const double *d_dev, double alpha, int maxit,
                                double rtol, int mode, double *h_out, double *hist, int *iters) {
    TRY(ready(c));
    if (!d_dev || !h_out || maxit < 0 || !(alpha >= 0) || !(rtol >= 0) ||
        (mode != SSX_MODE_PCG && mode != SSX_MODE_CG))
        return fail(c, SSX_ERR_ARG, "bad arguments");
    TRY(enter(c));
    std::vector<ShotRun> shots(1);
    shots[0].c = c;
    shots[0].alpha = alpha;
    shots[0].maxit = maxit;
    shots[0].rtol = rtol;
    shots[0].mode = mode;
    shots[0].d = d_dev;
    shots[0].h_out = h_out;
    shots[0].hist = hist;
    int rc = solve_batch(shots);
    if (iters) *iters = shots[0].iters;
    if (rc == SSX_OK) rc = shots[0].status;
    return leave(c, rc);
}

int ssx_solve_batch(ssx_ctx *const *ctxs, int n, const double *const *d_dev, const double *alphas,
                    int maxit, double rtol, int mode, double *const *h_out_dev, double *hist,
                    int *iters, int *status) {
    if (!ctxs || n < 1 || !d_dev || !alphas || !h_out_dev || maxit < 0 || !(rtol >= 0) ||
        (mode != SSX_MODE_PCG && mode != SSX_MODE_CG))
        return SSX_ERR_ARG;
    ssx_ctx *L = ctxs[0];
    if (!L) return SSX_ERR_ARG;
    for (int i = 0; i < n; i++) {
        if (!ctxs[i] || !d_dev[i] || !h_out_dev[i] || !(alphas[i] >= 0)) return fail(L, SSX_ERR_ARG, "bad shot arguments");
        TRY(ready(ctxs[i]));
        if (ctxs[i]->R != L->R) return fail(L, SSX_ERR_ARG, "all shots need the same space order");
        for (int j = 0; j < i; j++)
            if (ctxs[j] == ctxs[i]) return fail(L, SSX_ERR_ARG, "a context appears twice in the batch");
    }
    // order the lead stream after every shot's caller stream and internal stream
    auto c = L;
    for (int i = 0; i < n; i++) {
        CK(cudaEventRecord(ctxs[i]->ev_in, ctxs[i]->user));
        CK(cudaStreamWaitEvent(L->s, ctxs[i]->ev_in, 0));
        CK(cudaEventRecord(ctxs[i]->ev_in, ctxs[i]->s));
        CK(cudaStreamWaitEvent(L->s, ctxs[i]->ev_in, 0));
    }
    std::vector<ShotRun> shots(n);
    for (int i = 0; i < n; i++) {
        shots[i].c = ctxs[i];
        shots[i].alpha = alphas[i];
        shots[i].maxit = maxit;
        shots[i].rtol = rtol;
        shots[i].mode = mode;
        shots[i].d = d_dev[i];
        shots[i].h_out = h_out_dev[i];
        shots[i].hist = hist ? hist + (size_t)i * (maxit + 1) : nullptr;
    }
    int rc = solve_batch(shots);
    for (int i = 0; i < n; i++) {
        if (iters) iters[i] = shots[i].iters;
        if (status) status[i] = rc == SSX_OK ? shots[i].status : rc;
    }
    // every shot's later work (caller stream and internal stream) after the batch
    cudaEventRecord(L->ev_out, L->s);
    for (int i = 0; i < n; i++) {
        cudaStreamWaitEvent(ctxs[i]->user, L->ev_out, 0);
        cudaStreamWaitEvent(ctxs[i]->s, L->ev_out, 0);
    }
    return rc;
}

int ssx_point_source_data(ssx_ctx *c, double x_d, double z_d, const double *w, double *d_dev) {
    if (!c) return SSX_ERR_ARG;
    if (!c->have_model || !c->have_geom) return ready(c);
    if (!w || !d_dev) return fail(c, SSX_ERR_ARG, "null buffer");
    const double h = c->gd.h;
    const int ix = (int)std::lround(x_d / h);
    if (std::fabs(ix * h - x_d) > 1e-9) return fail(c, SSX_ERR_ARG, "x_d must fall on a grid column");
    Line pt{};
    TRY(make_line(c, c->full, z_d, ix, 1, 1.0 / h, &pt));
    TRY(enter(c));
    int rc = sim_fwd(c, c->full, pt, w, nullptr, c->rec, d_dev, nullptr, false);
    if (rc == SSX_OK) rc = check_sweeps(c);
    return leave(c, rc);
}

int ssx_set_sweep_mode(ssx_ctx *c, int mode) {
    if (!c) return SSX_ERR_ARG;
    if (mode == SSX_SWEEP_TEST_STALL) {
        c->stall_next = true;
        return SSX_OK;
    }
    if (mode != SSX_SWEEP_AUTO && mode != SSX_SWEEP_STEP && mode != SSX_SWEEP_PERSISTENT)
        return fail(c, SSX_ERR_ARG, "unknown sweep mode");
    c->sweep_mode = mode;
    reset_choices(c);
    return SSX_OK;
}

int ssx_set_test_hook(ssx_ctx *c, int hook, int k) {
    if (!c) return SSX_ERR_ARG;
    if (hook != SSX_HOOK_NONE && hook != SSX_HOOK_BREAKDOWN && hook != SSX_HOOK_NONFINITE)
        return fail(c, SSX_ERR_ARG, "unknown test hook");
    if (hook != SSX_HOOK_NONE && k < 0) return fail(c, SSX_ERR_ARG, "hook iteration must be >= 0");
    c->hook = hook;
    c->hook_k = k;
    return SSX_OK;
}

int ssx_set_tile_config(ssx_ctx *c, int cfg) {
    if (!c) return SSX_ERR_ARG;
    if (cfg < -1 || cfg >= kNumAllCfgs) return fail(c, SSX_ERR_ARG, "unknown tile configuration");
    c->forced_cfg = cfg;
    reset_choices(c);
    return SSX_OK;
}

int ssx_set_timing(ssx_ctx *c, int on) {
    if (!c) return SSX_ERR_ARG;
    c->timing = on != 0;
    return SSX_OK;
}

// Folds the recorded sweep events into the counters (synchronises).
static int resolve_events(ssx_ctx *c) {
    if (!c->ev_used) return SSX_OK;
    CK(cudaStreamSynchronize(c->s));
    for (size_t i = 0; i < c->ev_used; i++) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->evs[i].a, c->evs[i].b));
        c->st.sweep_ms += ms;
        c->st.timed_steps += c->evs[i].steps;
        c->st.timed_point_updates += c->evs[i].points;
        const int tag = c->evs[i].tag;
        if (tag >= 0 && tag < (int)c->phase_rows.size()) {
            c->phase_rows[tag].ms += ms;
            c->phase_rows[tag].steps += c->evs[i].steps;
        }
    }
    c->ev_used = 0;
    return SSX_OK;
}

int ssx_get_stats(ssx_ctx *c, ssx_stats *out) {
    if (!c || !out) return SSX_ERR_ARG;
    TRY(resolve_events(c));
    *out = c->st;
    const DGrid *gs[3] = {&c->full, &c->ss.g, &c->sr.g};
    for (int k = 0; k < 3; k++)
        for (int d = 0; d < 2; d++)
            out->tile_cfg[2 * k + d] = gs[k]->cfg[d] < 0 ? -1 : gs[k]->cfg[d] + (gs[k]->pers[d] ? 16 : 0);
    return SSX_OK;
}

int ssx_reset_stats(ssx_ctx *c) {
    if (!c) return SSX_ERR_ARG;
    if (c->ev_used) CK(cudaStreamSynchronize(c->s));
    c->ev_used = 0;
    c->st = ssx_stats{};
    c->phase_rows.clear();
    c->phase_row_of.clear();
    return SSX_OK;
}

int ssx_get_phase_stats(ssx_ctx *c, int k, char *name, int name_len, int *sweeps, int *tiles,
                        int *tile_cfg, int *chain, double *ms, long long *steps) {
    if (!c || k < 0 || !name || name_len < 1 || !sweeps || !tiles || !tile_cfg || !chain || !ms ||
        !steps)
        return SSX_ERR_ARG;
    TRY(resolve_events(c));
    if (k >= (int)c->phase_rows.size()) return SSX_ERR_ARG;
    const PhaseRow &r = c->phase_rows[k];
    snprintf(name, (size_t)name_len, "%s", r.name.c_str());
    *sweeps = r.sweeps;
    *tiles = r.tiles;
    *tile_cfg = r.cfg;
    *chain = r.chain;
    *ms = r.ms;
    *steps = r.steps;
    return SSX_OK;
}

int ssx_server_create(ssx_server **out, int space_order, size_t hbm_budget_bytes, void *stream) {
    if (!out || space_order < 2 || space_order > 8 || space_order % 2 || hbm_budget_bytes == 0)
        return SSX_ERR_ARG;
    *out = nullptr;
    ssx_server *sv = new ssx_server();
    sv->budget = hbm_budget_bytes;
    sv->order = space_order;
    ssx_grid_desc g{8, 8, 0.01, 1e-3, 1, space_order, 0};
    int rc = ssx_create(&sv->lead, &g, stream);
    if (rc != SSX_OK) {
        delete sv;
        return rc;
    }
    // requests come and go every few rounds: launch phases directly (no graph
    // capture per membership); tile configurations come from the phase tuner,
    // which keeps its choice per size class of batch for the process
    sv->lead->use_graphs = false;
    // working-set limit: four times the L2 size (on the full-size serving mix
    // 4x L2 served more requests per second than 1x, 2x or no limit)
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess)
        sv->cache_budget = 4 * (size_t)l2;
    *out = sv;
    return SSX_OK;
}

int ssx_server_set_cache_budget(ssx_server *sv, size_t bytes) {
    if (!sv) return SSX_ERR_ARG;
    sv->cache_budget = bytes;
    return SSX_OK;
}

int ssx_server_submit(ssx_server *sv, const ssx_grid_desc *grid, const ssx_geom_desc *geom,
                      const float *v_dev, double rho, const double *d_dev, double alpha, int maxit,
                      double rtol, int mode, double *h_out_dev, int *id_out) {
    if (!sv || !grid || !geom || !v_dev || !d_dev || !h_out_dev || !id_out || !(alpha >= 0) ||
        maxit < 0 || !(rtol >= 0) || (mode != SSX_MODE_PCG && mode != SSX_MODE_CG) || !(rho > 0))
        return SSX_ERR_ARG;
    if (grid->space_order != sv->order) {
        sv->err = "request space order differs from the server's";
        return SSX_ERR_ARG;
    }
    auto *q = new ssx_server::Req();
    q->id = sv->next_id++;
    q->g = *grid;
    q->m = *geom;
    q->v = v_dev;
    q->rho = rho;
    q->run.alpha = alpha;
    q->run.maxit = maxit;
    q->run.rtol = rtol;
    q->run.mode = mode;
    q->run.d = d_dev;
    q->run.h_out = h_out_dev;
    q->bytes = estimate_bytes(*grid, *geom);
    q->ws = field_bytes(*grid, *geom);
    q->t_submit = now_ms();
    sv->queue.push_back(q);
    sv->all[q->id] = q;
    *id_out = q->id;
    return SSX_OK;
}

int ssx_server_step(ssx_server *sv, int *n_active, int *n_queued) {
    if (!sv) return SSX_ERR_ARG;
    TRY(server_admit(sv));
    if (!sv->active.empty()) {
        ssx_ctx *L = sv->lead;
        ssx_ctx *c = L;
        CK(cudaEventRecord(L->ev_in, L->user));
        CK(cudaStreamWaitEvent(L->s, L->ev_in, 0));
        for (auto *q : sv->active) {   // after each request's own set-up work
            CK(cudaEventRecord(q->c->ev_in, q->c->s));
            CK(cudaStreamWaitEvent(L->s, q->c->ev_in, 0));
        }
        std::vector<ShotRun *> runs;
        for (auto *q : sv->active) runs.push_back(&q->run);
        sv->rounds++;
        sv->request_rounds += (long long)runs.size();
        int rc = engine_round(L, runs);
        if (rc != SSX_OK) {
            sv->err = L->err;
            return rc;
        }
        std::vector<ssx_server::Req *> keep;
        bool changed = false;
        for (auto *q : sv->active) {
            if (q->run.active()) {
                keep.push_back(q);
                continue;
            }
            TRY(engine_retire(L, q->run));
            CK(cudaStreamSynchronize(L->s));
            q->done = true;
            q->t_done = now_ms();
            ssx_destroy(q->c);
            q->c = nullptr;
            q->run.c = nullptr;
            sv->used -= q->bytes;
            sv->used_ws -= q->ws;
            changed = true;
        }
        sv->active.swap(keep);
        // phase tables of departed requests, and the graphs that read them
        if (changed) drop_graphs(L);
        CK(cudaEventRecord(L->ev_out, L->s));
        CK(cudaStreamWaitEvent(L->user, L->ev_out, 0));
    }
    if (n_active) *n_active = (int)sv->active.size();
    if (n_queued) *n_queued = (int)sv->queue.size();
    return SSX_OK;
}

int ssx_server_set_timing(ssx_server *sv, int on) {
    if (!sv) return SSX_ERR_ARG;
    return ssx_set_timing(sv->lead, on);
}

int ssx_server_get_stats(ssx_server *sv, ssx_stats *out, long long *rounds, long long *request_rounds) {
    if (!sv || !out) return SSX_ERR_ARG;
    const int rc = ssx_get_stats(sv->lead, out);
    if (rc != SSX_OK) {
        sv->err = sv->lead->err;
        return rc;
    }
    if (rounds) *rounds = sv->rounds;
    if (request_rounds) *request_rounds = sv->request_rounds;
    return SSX_OK;
}

int ssx_server_poll(ssx_server *sv, int id, int *done, int *status, int *iters, double *latency_ms,
                    double *queue_ms) {
    if (!sv) return SSX_ERR_ARG;
    auto it = sv->all.find(id);
    if (it == sv->all.end()) return SSX_ERR_ARG;
    ssx_server::Req *q = it->second;
    if (done) *done = q->done ? 1 : 0;
    if (status) *status = q->done ? q->run.status : SSX_OK;
    if (iters) *iters = q->run.iters;
    if (latency_ms) *latency_ms = q->done ? q->t_done - q->t_submit : 0.0;
    if (queue_ms) *queue_ms = q->t_admit > 0 ? q->t_admit - q->t_submit : 0.0;
    return SSX_OK;
}

int ssx_server_destroy(ssx_server *sv) {
    if (!sv) return SSX_ERR_ARG;
    if (sv->lead && sv->lead->s) cudaStreamSynchronize(sv->lead->s);
    for (auto &kv : sv->all) {
        if (kv.second->c) ssx_destroy(kv.second->c);
        delete kv.second;
    }
    if (sv->lead) ssx_destroy(sv->lead);
    delete sv;
    return SSX_OK;
}

const char *ssx_server_last_error(const ssx_server *sv) { return sv ? sv->err.c_str() : "null server"; }

}  // extern "C"
