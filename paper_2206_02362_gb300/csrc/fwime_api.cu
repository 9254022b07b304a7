// libfwime C ABI: argument validation, workspace planning, and the schedules
// that compose the kernels into the paper's operators (Barnier et al., Theory
// section, Eqs. 1, 7-9; Computational aspects: a shot is simulated on one GPU
// over the full FD domain, shots are independent).
//
// Schedules.  Shots are processed in batches of S advanced together (one
// launch per kernel per time step covers the whole batch).  Time is cut into
// segments of K steps:
//   * forward-type operators (f, B, B~, T) run segment by segment: the
//     background wavefield's D2t over K steps goes to a ring, one scatter
//     launch turns the whole ring (K x S pairs) into secondary sources, then
//     the scattered field steps through the segment;
//   * adjoint-type operators (B*, B~*, T*, gradient) store the background (and
//     scattered) state at every segment start during a forward sweep, then walk
//     the segments backwards: recompute the segment's D2t fields into rings,
//     step the adjoint fields down through it, and reduce the imaging
//     conditions over the segment's K x S pairs in one launch.
// The adjoint wavefield uses mu = c g lambda, which obeys the forward recursion
// run backwards, so forward and adjoint share the stencil kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/fwime.h"
#include "fwime_internal.h"
#include "fwime_kernels.cuh"

using namespace fwk;

namespace {

struct Graph {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
};

}  // namespace

struct fwime_ctx {
    fwime_grid g{};
    int nshot = 0, nrec = 0;
    std::vector<int> src_iz, src_ix, rec_iz, rec_ix;
    int NZ = 0, NX = 0, NXP = 0, o = 0;
    long long P = 0;
    cudaStream_t st = nullptr;
    size_t max_ws = 0;
    int device = 0;
    // options
    int opt_S = 0, opt_K = 0, opt_plain = 0, opt_graph = 0, opt_host_io = 0, opt_zchunk = 0, opt_reuse_bg = 0;
    int opt_tlag = 0;               // > 0: B~ / B~* extend with time lags spaced opt_tlag steps
    int opt_fs = 0;                 // 1: free surface at the top physical row
    // background-wavefield checkpoints of every shot, [nseg][2][nshot][P], written by B and B~ and
    // read by B* and B~* on the same v, w (FWIME_OPT_REUSE_BACKGROUND)
    struct BgCache {
        float *buf = nullptr;
        size_t bytes = 0;
        bool valid = false;
        const float *v = nullptr, *w = nullptr;
        int K = 0;
    } bg;
    bool bg_written = false;        // set by the last enqueued B / B~ that filled the cache
    // state the forward half of the gradient leaves for its adjoint half (fwime_gradient_forward /
    // fwime_gradient_backward): segment-start states of the background and scattered fields of every
    // shot, [nseg][4][nshot][P], then the residual r = f + B~ p~ - d_obs, [nshot][nt][nrec]
    struct GradState {
        float *buf = nullptr;
        size_t bytes = 0;
        bool valid = false;
        const float *v = nullptr, *w = nullptr, *pt = nullptr;
        int K = 0;
    } gs;
    bool bg_used = false;           // the last call started from the cache
    long long launches = 0;
    int last_S = 0;                 // shots per batch the last planned operator call used
    // persistent device memory
    int *d_src_off = nullptr, *d_rec_off = nullptr, *d_status = nullptr;
    double *d_J = nullptr, *d_part = nullptr, *h_J = nullptr;
    int *h_status = nullptr;
    void *small = nullptr;          // one stream-ordered block: J, partials, status, offsets
    std::vector<int> h_off;         // host copy of the offsets (source of the async upload)
    // receiver injection map for the adjoint steps: rows [inj_lo, inj_hi) x NXP -> first receiver at the
    // point or -1, then the chain of further receivers at the same point (host copy and device copy)
    std::vector<int> h_inj;
    int *d_inj_map = nullptr, *d_inj_next = nullptr;
    int inj_lo = 0, inj_hi = 0;
    double *user_J = nullptr;
    double *vp_hist_dev = nullptr, *vp_hist_user = nullptr;   // VP objective history (device, caller's host)
    int vp_hist_n = 0;
    // workspace arena
    char *ws = nullptr;
    size_t ws_bytes = 0;
    std::map<std::string, Graph> graphs;
    bool capturing = false;
    // per-launch CUDA-event profiling (FWIME_OPT_PROFILE)
    int opt_profile = 0;
    struct Pend { int ev; int kind; double bytes; };
    std::vector<cudaEvent_t> ev;
    std::vector<Pend> pend;
    double prof_ms[5] = {0, 0, 0, 0, 0}, prof_bytes[5] = {0, 0, 0, 0, 0};
    long long prof_n[5] = {0, 0, 0, 0, 0};
    int last_err = 0;
    char err[320] = {0};
    Server *srv = nullptr;          // a server context (fwime_server_create): no grid, no operators
};

namespace fwk {
fwime_ctx *ctx_for_server(Server *srv)
{
    fwime_ctx *x = new fwime_ctx();
    x->srv = srv;
    return x;
}
Server *ctx_server(const fwime_ctx *x) { return x ? x->srv : nullptr; }
}  // namespace fwk

// operator entry points refuse a server context
#define NOT_SERVER(x)                                                                                  \
    do {                                                                                               \
        if ((x)->srv) return fail((x), FWIME_EINVAL, "a server context takes requests (fwime_submit), not operators"); \
    } while (0)

// ------------------------------------------------------------------ helpers

// A process-wide pinned block handing every context two 8-byte slots (objective and
// status read-back) so that creating a context never calls a synchronising host
// allocator.  Slots are reused round-robin.
static double *pinned_slot()
{
    static double *pool = nullptr;
    static std::atomic<unsigned> next{0};
    static std::once_flag once;
    constexpr unsigned NSLOT = 8192;
    std::call_once(once, [] {
        if (cudaMallocHost(reinterpret_cast<void **>(&pool), 2 * NSLOT * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            pool = nullptr;
        }
    });
    if (!pool) return nullptr;
    return pool + 2 * (next.fetch_add(1) % NSLOT);
}

static int fail(fwime_ctx *x, int code, const char *fmt, ...)
{
    if (x) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(x->err, sizeof(x->err), fmt, ap);
        va_end(ap);
        x->last_err = code;
    }
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(x, FWIME_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define TRY(call)                                                                                  \
    do {                                                                                           \
        int r_ = (call);                                                                           \
        if (r_ != FWIME_OK) return r_;                                                             \
    } while (0)

// Event pair around one launch when profiling; `bytes` are the launch's algorithmic bytes.
static int prof_begin(fwime_ctx *x, int &slot)
{
    slot = -1;
    if (!x->opt_profile) return FWIME_OK;
    const size_t need = 2 * (x->pend.size() + 1);
    while (x->ev.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        x->ev.push_back(e);
    }
    slot = (int)(2 * x->pend.size());
    CK(cudaEventRecord(x->ev[slot], x->st));
    return FWIME_OK;
}

static int prof_end(fwime_ctx *x, int slot, int kind, double bytes)
{
    if (slot < 0) return FWIME_OK;
    CK(cudaEventRecord(x->ev[slot + 1], x->st));
    x->pend.push_back({slot, kind, bytes});
    return FWIME_OK;
}

static int prof_collect(fwime_ctx *x)
{
    if (x->pend.empty()) return FWIME_OK;
    CK(x->st ? cudaStreamSynchronize(x->st) : cudaDeviceSynchronize());
    for (const auto &p : x->pend) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, x->ev[p.ev], x->ev[p.ev + 1]));
        x->prof_ms[p.kind] += ms;
        x->prof_bytes[p.kind] += p.bytes;
        x->prof_n[p.kind] += 1;
    }
    x->pend.clear();
    return FWIME_OK;
}

// a kernel launch: counts it and, when profiling, brackets it with events
#define LAUNCH(kind, bytes, call)                                                                  \
    do {                                                                                           \
        int slot_;                                                                                 \
        TRY(prof_begin(x, slot_));                                                                 \
        x->launches++;                                                                             \
        CK(call);                                                                                  \
        TRY(prof_end(x, slot_, (kind), (bytes)));                                                  \
    } while (0)

static int auto_K(int nt)
{
    int K = (int)std::lround(std::sqrt((double)std::max(nt - 1, 1)));
    return std::min(std::max(K, 8), 128);
}

// Floats of workspace: model part (independent of S) and per-shot part.
struct Sizes {
    size_t model = 0, per_shot = 0, staging = 0;
};

static size_t al(size_t n) { return (n + 63) & ~(size_t)63; }   // 256-byte granules

// time-lag extension: shifts reach Hs = 2 hm lag steps either way; the background D2t ring holds K + 2 Hs
// steps; the adjoint recomputes the background in blocks [j K - Hs, (j+1) K - Hs), j = 0 .. tlag_blocks - 1
static int tlag_Hs(const fwime_grid &g, int lag) { return (g.nh - 1) * lag; }
static int tlag_blocks(const fwime_grid &g, int K, int lag) { return (g.nt - 2 + tlag_Hs(g, lag)) / K + 1; }

static Sizes op_sizes(const fwime_grid &g, int nshot, int nrec, long long P, int NZ, int NXP, int op, int K,
                      bool host_io, bool no_ckpt = false, int tlag = 0)
{
    Sizes s;
    const size_t nh = g.nh, nseg = (size_t)((g.nt - 1 + K - 1) / K), R = K + 2;
    if (tlag > 0 && op != FWIME_OP_FORWARD && op != FWIME_OP_BORN && op != FWIME_OP_BORN_ADJ) {
        const size_t Hs = tlag_Hs(g, tlag), RD = (size_t)K + 2 * Hs, NB = tlag_blocks(g, K, tlag);
        s.model = al(P) * 2 + al(NZ) + al(NXP);
        size_t f = 0;
        switch (op) {
        case FWIME_OP_BORN_EXT: s.model += al(nh * P); f = 4 + RD + K; break;
        case FWIME_OP_BORN_EXT_ADJ: s.model += al(nh * P); f = 2 + RD + R + 2 * NB; break;
        case FWIME_OP_TOMO: s.model += 2 * al(nh * P) + al(P); f = 8 + 2 * RD + 2 * K; break;
        default:   // T*, gradient, objective
            s.model += 2 * al(nh * P) + al(P);
            f = 4 + RD + 2 * (size_t)K + (RD + 2) + 2 * R + 2 * NB + 2 * nseg;
        }
        s.per_shot = f * (size_t)P;
        if (op == FWIME_OP_GRADIENT || op == FWIME_OP_OBJECTIVE) s.per_shot += (size_t)g.nt * nrec;
        if (host_io) {
            const size_t nd = (size_t)nshot * g.nt * nrec, nm = (size_t)g.nz * g.nx;
            s.staging = al(nm) + al((size_t)nshot * g.nt) + 2 * al(nd) + al(nh * nm) + al(nm) + al(nh * nm);
        }
        return s;
    }
    s.model = al(P) * 2 + al(NZ) + al(NXP);   // c, bpad, gz, gx
    size_t f = 0;
    switch (op) {
    case FWIME_OP_FORWARD: f = 2; break;
    case FWIME_OP_BORN: s.model += al(P); f = 5; break;
    case FWIME_OP_BORN_EXT: s.model += al(nh * P); f = 4 + 2 * K; break;
    case FWIME_OP_BORN_ADJ: s.model += al(P); f = 2 + K + R + (no_ckpt ? 0 : 2 * nseg); break;
    case FWIME_OP_BORN_EXT_ADJ: s.model += al(nh * P); f = 2 + K + R + (no_ckpt ? 0 : 2 * nseg); break;
    case FWIME_OP_TOMO: s.model += 2 * al(nh * P) + al(P); f = 8 + 4 * K; break;
    case FWIME_OP_TOMO_ADJ:
    case FWIME_OP_GRADIENT: s.model += 2 * al(nh * P) + 2 * al(P); f = 4 + 3 * K + 3 * R + (no_ckpt ? 0 : 4 * nseg); break;
    case FWIME_OP_OBJECTIVE: s.model += 2 * al(nh * P) + 2 * al(P); f = 4 + 2 * K; break;
    default: break;
    }
    s.per_shot = f * (size_t)P;
    // gradient and objective predict the data into the workspace, unless the context's gradient state holds it
    if ((op == FWIME_OP_GRADIENT || op == FWIME_OP_OBJECTIVE) && !no_ckpt) s.per_shot += (size_t)g.nt * nrec;
    if (host_io) {
        const size_t nd = (size_t)nshot * g.nt * nrec, nm = (size_t)g.nz * g.nx;
        s.staging = al(nm) + al((size_t)nshot * g.nt) + 2 * al(nd) + al(nh * nm) + al(nm) + al(nh * nm);
    }
    return s;
}

static int validate(const fwime_grid *g, const fwime_geom *geo, fwime_ctx *x)
{
    if (!g || !geo) return fail(x, FWIME_EINVAL, "null grid or geometry");
    if (g->nz < 1 || g->nx < 1 || g->sponge < 0 || g->nt < 2)
        return fail(x, FWIME_EINVAL, "grid sizes: nz=%d nx=%d sponge=%d nt=%d", g->nz, g->nx, g->sponge, g->nt);
    if (g->nh < 1 || g->nh % 2 == 0 || g->nh > MAX_NH)
        return fail(x, FWIME_EINVAL, "nh=%d must be odd, 1..%d", g->nh, MAX_NH);
    if (!(g->dx > 0.f) || !(g->dz > 0.f) || !(g->dt > 0.f)) return fail(x, FWIME_EINVAL, "spacings must be > 0");
    if (geo->nshot < 1 || geo->nrec < 1) return fail(x, FWIME_EINVAL, "nshot=%d nrec=%d", geo->nshot, geo->nrec);
    if (!geo->src_iz || !geo->src_ix || !geo->rec_iz || !geo->rec_ix) return fail(x, FWIME_EINVAL, "null geometry");
    for (int s = 0; s < geo->nshot; ++s)
        if (geo->src_iz[s] < 0 || geo->src_iz[s] >= g->nz || geo->src_ix[s] < 0 || geo->src_ix[s] >= g->nx)
            return fail(x, FWIME_EINVAL, "source %d at (%d,%d) outside the grid", s, geo->src_iz[s], geo->src_ix[s]);
    for (int r = 0; r < geo->nrec; ++r)
        if (geo->rec_iz[r] < 0 || geo->rec_iz[r] >= g->nz || geo->rec_ix[r] < 0 || geo->rec_ix[r] >= g->nx)
            return fail(x, FWIME_EINVAL, "receiver %d at (%d,%d) outside the grid", r, geo->rec_iz[r], geo->rec_ix[r]);
    return FWIME_OK;
}

// ------------------------------------------------------------ workspace

struct WS {
    int S = 1, K = 8, nseg = 1, R = 10;
    // model
    float *c, *bpad, *gz, *gx, *coef, *W, *W2, *ptp, *acc1, *acc2;
    // per batch
    float *f[8];
    float *ring[6];    // rings of K slots (ring[0..3]) and of R slots (ring[3..5] in adjoint ops)
    float *ckpt, *pred;
    // host-io staging
    float *sv, *sw, *sd1, *sd2, *sm1, *sdv, *smo;
};

static int plan(fwime_ctx *x, int op, WS &w, bool no_ckpt = false)
{
    w.K = x->opt_K > 0 ? x->opt_K : auto_K(x->g.nt);
    // time lags: segments of at least 4 Hs steps keep the lag halo (2 Hs samples per segment, read once per
    // residue class) at half the segment's own K samples or less
    if (x->opt_tlag > 0 && x->opt_K == 0) w.K = std::max(w.K, 4 * tlag_Hs(x->g, x->opt_tlag));
    w.K = std::min(w.K, x->g.nt - 1);
    w.K = std::max(w.K, 1);
    w.nseg = (x->g.nt - 1 + w.K - 1) / w.K;
    w.R = w.K + 2;
    Sizes sz = op_sizes(x->g, x->nshot, x->nrec, x->P, x->NZ, x->NXP, op, w.K, x->opt_host_io != 0, no_ckpt,
                        x->opt_tlag);
    size_t budget = x->max_ws;
    if (budget == 0 && x->capturing) budget = x->ws_bytes;   // the workspace was planned before capture
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        CK(cudaMemGetInfo(&fr, &tot));
        budget = x->ws_bytes + fr;
        budget = budget > ((size_t)2 << 30) ? budget - ((size_t)2 << 30) : budget / 2;   // keep 2 GB slack
    }
    // a default time-lag segment of 4 Hs that does not fit one shot falls back to 2 Hs (the halo then
    // equals the segment's own samples; the kernels stay correct for any K)
    if (x->opt_tlag > 0 && x->opt_K == 0 && w.K > 2 * tlag_Hs(x->g, x->opt_tlag) &&
        (sz.model + sz.staging + sz.per_shot) * sizeof(float) > budget) {
        w.K = std::max(std::min(std::max(auto_K(x->g.nt), 2 * tlag_Hs(x->g, x->opt_tlag)), x->g.nt - 1), 1);
        w.nseg = (x->g.nt - 1 + w.K - 1) / w.K;
        w.R = w.K + 2;
        sz = op_sizes(x->g, x->nshot, x->nrec, x->P, x->NZ, x->NXP, op, w.K, x->opt_host_io != 0, no_ckpt,
                      x->opt_tlag);
    }
    const size_t fixed = (sz.model + sz.staging) * sizeof(float);
    const size_t per = sz.per_shot * sizeof(float);
    int S;
    if (x->opt_plain) S = 1;
    else if (x->opt_S > 0) S = std::min(x->opt_S, x->nshot);
    else {
        if (fixed + per > budget) S = 1;
        else S = (int)std::min<size_t>((size_t)x->nshot, (budget - fixed) / per);
        // as many batches as memory forces, of equal size: a short last batch runs its launches at a
        // fraction of the work for the same per-launch overheads
        S = std::max(S, 1);
        const int nb = (x->nshot + S - 1) / S;
        S = (x->nshot + nb - 1) / nb;
    }
    w.S = std::max(S, 1);
    x->last_S = w.S;
    const size_t need = fixed + per * (size_t)w.S + 4096;
    if (x->max_ws && need > x->max_ws)
        return fail(x, FWIME_ENOMEM, "operator needs %zu bytes for S=%d, K=%d; budget %zu", need, w.S, w.K, x->max_ws);
    if (need > x->ws_bytes) {
        if (x->capturing) return fail(x, FWIME_EBUSY, "workspace growth during graph capture");
        // stream-ordered (re)allocation: no device-wide synchronisation, so contexts of other
        // streams keep running while this one grows
        if (x->ws) {
            for (auto &kv : x->graphs) cudaGraphExecDestroy(kv.second.exec);
            x->graphs.clear();
            CK(cudaFreeAsync(x->ws, x->st));
            x->ws = nullptr;
            x->ws_bytes = 0;
        }
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&x->ws), need, x->st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(x, FWIME_ENOMEM, "cudaMallocAsync(%zu): %s", need, cudaGetErrorString(e));
        }
        x->ws_bytes = need;
    }
    // carve
    float *p = reinterpret_cast<float *>(x->ws);
    auto take = [&](size_t n) { float *r = p; p += al(n); return r; };
    const long long P = x->P;
    const size_t nh = x->g.nh;
    // host-I/O staging first: the same addresses for every operator (a staged v or w keeps its address
    // from one call to the next as long as the arena is not reallocated)
    w.sv = w.sw = w.sd1 = w.sd2 = w.sm1 = w.sdv = w.smo = nullptr;
    if (x->opt_host_io) {
        const size_t nd = (size_t)x->nshot * x->g.nt * x->nrec, nm = (size_t)x->g.nz * x->g.nx;
        w.sv = take(nm); w.sw = take((size_t)x->nshot * x->g.nt); w.sd1 = take(nd); w.sd2 = take(nd);
        w.sm1 = take(nh * nm); w.sdv = take(nm); w.smo = take(nh * nm);
    }
    w.c = take(P); w.bpad = take(P); w.gz = take(x->NZ); w.gx = take(x->NXP);
    w.coef = w.W = w.W2 = w.ptp = w.acc1 = w.acc2 = nullptr;
    switch (op) {
    case FWIME_OP_BORN: w.coef = take(P); break;
    case FWIME_OP_BORN_EXT: w.W = take(nh * P); break;
    case FWIME_OP_BORN_ADJ: w.acc1 = take(P); break;
    case FWIME_OP_BORN_EXT_ADJ: w.acc1 = take(nh * P); break;
    case FWIME_OP_TOMO: w.W = take(nh * P); w.W2 = take(nh * P); w.coef = take(P); break;
    case FWIME_OP_TOMO_ADJ:
    case FWIME_OP_GRADIENT:
    case FWIME_OP_OBJECTIVE: w.W = take(nh * P); w.acc1 = take(P); w.acc2 = take(nh * P); break;
    default: break;
    }
    const size_t SP = (size_t)w.S * P;
    for (auto &q : w.f) q = nullptr;
    for (auto &q : w.ring) q = nullptr;
    w.ckpt = w.pred = nullptr;
    int nf = 0, nk = 0, nr = 0, nck = 0;
    if (x->opt_tlag > 0 && op != FWIME_OP_FORWARD && op != FWIME_OP_BORN && op != FWIME_OP_BORN_ADJ) {
        const size_t RD = (size_t)w.K + 2 * tlag_Hs(x->g, x->opt_tlag), NB = tlag_blocks(x->g, w.K, x->opt_tlag);
        const size_t K = w.K, R = w.R;
        switch (op) {
        case FWIME_OP_BORN_EXT:   // fields q0, dq; ring[0] D2t q0 (K + 2 Hs), ring[1] scatter output (K)
            for (int i = 0; i < 4; ++i) w.f[i] = take(SP);
            w.ring[0] = take(RD * SP); w.ring[1] = take(K * SP);
            break;
        case FWIME_OP_BORN_EXT_ADJ:   // ring[0] D2t q0, ring[1] adjoint field (K + 2); block checkpoints
            for (int i = 0; i < 2; ++i) w.f[i] = take(SP);
            w.ring[0] = take(RD * SP); w.ring[1] = take(R * SP);
            w.ckpt = take(NB * 2 * SP);
            break;
        case FWIME_OP_TOMO:   // rings: D2t q0, D2t dq0 (K + 2 Hs), scatter output, D2t dqs (K)
            for (int i = 0; i < 8; ++i) w.f[i] = take(SP);
            w.ring[0] = take(RD * SP); w.ring[1] = take(RD * SP); w.ring[2] = take(K * SP); w.ring[3] = take(K * SP);
            break;
        default:   // T*, gradient, objective: D2t q0, scatter output, D2t dqs, mu (K + 2 Hs + 2), z, mu2
            for (int i = 0; i < 4; ++i) w.f[i] = take(SP);
            w.ring[0] = take(RD * SP); w.ring[1] = take(K * SP); w.ring[2] = take(K * SP);
            w.ring[3] = take((RD + 2) * SP); w.ring[4] = take(R * SP); w.ring[5] = take(R * SP);
            w.ckpt = take((NB + (size_t)w.nseg) * 2 * SP);
            if (op == FWIME_OP_GRADIENT || op == FWIME_OP_OBJECTIVE) w.pred = take((size_t)w.S * x->g.nt * x->nrec);
        }
        if ((char *)p > x->ws + x->ws_bytes) return fail(x, FWIME_ENOMEM, "workspace layout overflow");
        return FWIME_OK;
    }
    switch (op) {
    case FWIME_OP_FORWARD: nf = 2; break;
    case FWIME_OP_BORN: nf = 5; break;
    case FWIME_OP_BORN_EXT: nf = 4; nk = 2; break;
    case FWIME_OP_BORN_ADJ:
    case FWIME_OP_BORN_EXT_ADJ: nf = 2; nk = 1; nr = 1; nck = no_ckpt ? 0 : 2; break;
    case FWIME_OP_TOMO: nf = 8; nk = 4; break;
    case FWIME_OP_OBJECTIVE: nf = 4; nk = 2; break;
    default: nf = 4; nk = 3; nr = 3; nck = no_ckpt ? 0 : 4; break;
    }
    for (int i = 0; i < nf; ++i) w.f[i] = take(SP);
    for (int i = 0; i < nk; ++i) w.ring[i] = take((size_t)w.K * SP);
    for (int i = 0; i < nr; ++i) w.ring[nk + i] = take((size_t)w.R * SP);
    if (nck) w.ckpt = take((size_t)w.nseg * nck * SP);
    if ((op == FWIME_OP_GRADIENT || op == FWIME_OP_OBJECTIVE) && !no_ckpt)
        w.pred = take((size_t)w.S * x->g.nt * x->nrec);
    if ((char *)p > x->ws + x->ws_bytes) return fail(x, FWIME_ENOMEM, "workspace layout overflow");
    return FWIME_OK;
}

// --------------------------------------------------------------- launches

struct Run {
    fwime_ctx *x;
    WS w;
    int zchunk, nstrip, nchunk;
    PropArgs base{};
};

static void init_run(fwime_ctx *x, Run &r, int S)
{
    r.x = x;
    const int rows = x->NZ - 8;
    r.nstrip = (x->NXP + STRIP - 1) / STRIP;
    int zc = x->opt_zchunk;
    if (zc <= 0) {
        const long long target = 152LL * 32;   // resident warps to aim for
        long long per = (long long)r.nstrip * std::max(S, 1);
        long long nchunk_t = std::max<long long>(1, (target + per - 1) / per);
        zc = (int)((rows + nchunk_t - 1) / nchunk_t);
        zc = std::min(std::max(zc, 8), 256);
    }
    r.zchunk = zc;
    r.nchunk = (rows + zc - 1) / zc;
    PropArgs &a = r.base;
    std::memset(&a, 0, sizeof(a));
    a.NZ = x->NZ; a.NXP = x->NXP; a.zchunk = r.zchunk; a.nstrip = r.nstrip; a.nchunk = r.nchunk; a.P = x->P;
    const double A8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
    for (int k = 0; k < 5; ++k) {
        a.ax[k] = (float)(A8[k] / ((double)x->g.dx * x->g.dx));
        a.az[k] = (float)(A8[k] / ((double)x->g.dz * x->g.dz));
    }
    a.inv_dt2 = (float)(1.0 / ((double)x->g.dt * x->g.dt));
    a.src_scale = (float)(1.0 / ((double)x->g.dx * x->g.dz));
    a.zs_lo = x->o; a.zs_hi = x->o + x->g.nz;
}

// Receivers of a stencil launch's input field, recorded by the launch itself: row d of the data (=, or +=).
struct RecTo {
    float *d = nullptr;
    int acc = 0;
};

// Residual injected at the receivers into a (plain) stencil launch's output: row `val` of the data.
struct InjFrom {
    const float *val = nullptr;
};

static int prop(Run &r, int Sb, const float *cur, const float *prev, float *out, float *d2, const float *wsrc,
                int src_shot0, const float *f0 = nullptr, float a0 = 0.f, const float *f1 = nullptr, float a1 = 0.f,
                const float *f2 = nullptr, float a2 = 0.f, const float *coef = nullptr, const float *fc = nullptr,
                RecTo rec = RecTo{}, InjFrom inj = InjFrom{})
{
    fwime_ctx *x = r.x;
    PropArgs a = r.base;
    a.c = r.w.c; a.gz = r.w.gz; a.gx = r.w.gx;
    a.cur = cur; a.prev = prev; a.out = out; a.d2 = d2;
    if (wsrc) {
        a.src_off = x->d_src_off + src_shot0;
        a.src_amp = wsrc;
        a.src_stride = x->g.nt;
    }
    a.f0 = f0; a.a0 = a0; a.f1 = f1; a.a1 = a1; a.f2 = f2; a.a2 = a2; a.coef = coef; a.fc = fc;
    if (rec.d) {
        a.rec_off = x->d_rec_off; a.rec_d = rec.d; a.rec_dstride = (long long)x->g.nt * x->nrec;
        a.nrec = x->nrec; a.rec_acc = rec.acc;
    }
    if (inj.val) {
        a.inj_map = x->d_inj_map; a.inj_next = x->d_inj_next; a.inj_val = inj.val;
        a.inj_vstride = (long long)x->g.nt * x->nrec; a.inj_lo = x->inj_lo; a.inj_hi = x->inj_hi;
    }
    // compulsory bytes: per shot-point read q^n, q^{n-1}, write q^{n+1}, and per point once per launch
    // the shared c, over the padded grid; D2t out and the local source fields (and coef) over the
    // physical rows only (zero elsewhere, not needed there)
    const double pts = (double)x->NZ * x->NX, spts = (double)x->g.nz * x->NX;
    const double srcb = (d2 ? 4 : 0) + 4.0 * ((f0 != nullptr) + (f1 != nullptr) + (f2 != nullptr)) + (fc ? 4 : 0);
    const double recb = (rec.d ? (double)Sb * x->nrec * (rec.acc ? 12.0 : 8.0) : 0.0) +
                        (inj.val ? (double)Sb * x->nrec * 4.0 : 0.0);
    LAUNCH(FWIME_K_PROP, pts * (Sb * 12.0 + 4.0) + spts * (Sb * srcb + (coef ? 4.0 : 0.0)) + recb,
           launch_prop(a, Sb, x->st));
    if (x->opt_fs)
        LAUNCH(FWIME_K_OTHER, (double)Sb * x->NXP * (d2 ? 44.0 : 40.0),
               launch_free_surface(out, d2, Sb, x->P, x->NXP, x->o, x->st));
    return FWIME_OK;
}

static int record(Run &r, int Sb, const float *f1, const float *f2, float *d, int accumulate)
{
    fwime_ctx *x = r.x;
    PointsArgs a{};
    a.nrec = x->nrec; a.P = x->P; a.rec_off = x->d_rec_off;
    a.f1 = f1; a.f2 = f2; a.d = d; a.dstride = (long long)x->g.nt * x->nrec; a.accumulate = accumulate;
    LAUNCH(FWIME_K_POINTS, (double)Sb * x->nrec * (8.0 + (f2 ? 4 : 0) + (accumulate ? 4 : 0)),
           launch_points(a, Sb, x->st));
    return FWIME_OK;
}

// One adjoint time step with the residual's injection at the receivers folded into the stencil launch
// (the transpose of recording; the same arithmetic as a separate injection after the step), and
// optionally the D2t of its output, injection included
static int adj_step(Run &r, int Sb, const float *cur, const float *prev, float *out, const float *val,
                    float *d2 = nullptr)
{
    return prop(r, Sb, cur, prev, out, d2, nullptr, 0, nullptr, 0.f, nullptr, 0.f, nullptr, 0.f, nullptr,
                nullptr, RecTo{}, InjFrom{val});
}

static RingRef ringref(const float *base, long long slot_stride, int mod, int shift)
{
    RingRef rr;
    rr.base = base; rr.slot_stride = slot_stride; rr.mod = mod; rr.shift = shift;
    return rr;
}

// x-range of points a scatter can reach: physical columns +- hm, within the active region
static void ext_cols(fwime_ctx *x, int &lo, int &hi)
{
    const int hm = (x->g.nh - 1) / 2;
    lo = std::max(4, x->o - hm);
    hi = std::min(x->NX - 4, x->o + x->g.nx + hm);
}

static int scatter(Run &r, int Sb, int n0, int kk, const float *W, RingRef in, RingRef out, int sigma, int accumulate)
{
    fwime_ctx *x = r.x;
    ExtArgs a{};
    a.NXP = x->NXP; a.nh = x->g.nh; a.hm = (x->g.nh - 1) / 2; a.S = Sb; a.npair = kk * Sb; a.n0 = n0; a.P = x->P;
    a.z_lo = x->o; a.z_hi = x->o + x->g.nz;
    ext_cols(x, a.x_lo, a.x_hi);   // the launcher may start a few columns earlier (zero weights there)
    a.sigma = sigma; a.W = W; a.in = in; a.outr = out; a.accumulate = accumulate;
    const double pts = (double)x->g.nz * (a.x_hi - a.x_lo);
    LAUNCH(FWIME_K_SCATTER, pts * ((double)a.npair * (8.0 + (accumulate ? 4 : 0)) + 4.0 * x->g.nh),
           launch_scatter(a, x->st));
    return FWIME_OK;
}

// img_local (IMG_EXT only): the same launch also adds the IMG_LOCAL terms of M2 and Ds into it
static int image(Run &r, int Sb, int n0, int kk, int mode, RingRef D, RingRef L, RingRef M2, RingRef Ds, float alpha,
                 const float *pt, float *img, float *img_local = nullptr)
{
    fwime_ctx *x = r.x;
    ImgArgs a{};
    a.NXP = x->NXP; a.nh = x->g.nh; a.hm = (x->g.nh - 1) / 2; a.S = Sb; a.npair = kk * Sb; a.n0 = n0; a.P = x->P;
    a.z_lo = x->o; a.z_hi = x->o + x->g.nz; a.x_lo = x->o; a.x_hi = x->o + x->g.nx;   // the physical columns
    a.D = D; a.L = L; a.M2 = M2; a.Ds = Ds; a.alpha = alpha; a.pt = pt; a.img = img; a.img_local = img_local;
    const double pts = (double)x->g.nz * x->g.nx;
    const double per = 8.0 + (M2.base ? 4 : 0) + (Ds.base ? 4 : 0);
    const double once = mode == IMG_EXT ? 8.0 * x->g.nh + (img_local ? 8.0 : 0.0)
                                        : (mode == IMG_CONTRACT ? 8.0 + 4.0 * x->g.nh : 8.0);
    LAUNCH(FWIME_K_IMAGE, pts * ((double)a.npair * per + once), launch_image(a, mode, x->st));
    return FWIME_OK;
}

static int zero(fwime_ctx *x, void *p, size_t bytes)
{
    if (bytes == 0) return FWIME_OK;
    CK(cudaMemsetAsync(p, 0, bytes, x->st));
    return FWIME_OK;
}

static int copyf(fwime_ctx *x, float *dst, const float *src, size_t n)
{
    LAUNCH(FWIME_K_OTHER, 8.0 * n, launch_copy_fields(dst, src, (long long)n, x->st));
    return FWIME_OK;
}

static int prep_model(fwime_ctx *x, Run &r, const float *v)
{
    PrepArgs a{};
    a.nz = x->g.nz; a.nx = x->g.nx; a.o = x->o; a.NZ = x->NZ; a.NX = x->NX; a.NXP = x->NXP; a.W = x->g.sponge;
    a.dt = x->g.dt;
    a.cfl_limit2 = cfl_vmax2(x->g.dt, x->g.dx, x->g.dz);
    a.v = v; a.c = r.w.c; a.gz = r.w.gz; a.gx = r.w.gx; a.bpad = r.w.bpad; a.status = x->d_status;
    a.fs = x->opt_fs;
    LAUNCH(FWIME_K_OTHER, 12.0 * x->NZ * x->NXP, launch_prep(a, x->st));
    return FWIME_OK;
}

// ------------------------------------------------------------- schedules

// ---------------------------------------------------------------- background checkpoint cache
// B and B~ propagate the background wavefield forward anyway; with FWIME_OPT_REUSE_BACKGROUND they also
// copy its state (q^n0, q^n0-1) at every segment start n0 = j K, for every shot, into a context-owned
// array [nseg][2][nshot][P].  B* and B~* on the same v and w then start their backward sweeps from these
// states instead of running their own checkpointing sweep (one propagation fewer per call; the states are
// those the sweep would compute).

static int seg_K(const fwime_ctx *x)
{
    int K = x->opt_K > 0 ? x->opt_K : auto_K(x->g.nt);
    return std::max(std::min(K, x->g.nt - 1), 1);
}

static size_t bg_bytes(const fwime_ctx *x, int K)
{
    const size_t nseg = (size_t)((x->g.nt - 1 + K - 1) / K);
    return nseg * 2 * (size_t)x->nshot * (size_t)x->P * sizeof(float);
}

// Makes room for the cache; false when it does not fit (the call then runs without it).
static bool bg_reserve(fwime_ctx *x, int K)
{
    const size_t need = bg_bytes(x, K);
    if (x->bg.buf && x->bg.bytes >= need) return true;
    if (x->capturing) return false;
    if (x->max_ws && x->ws_bytes + need > x->max_ws) return false;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (need + ((size_t)4 << 30) > fr + x->bg.bytes) return false;   // leave room for the operator's workspace
    if (x->bg.buf) cudaFreeAsync(x->bg.buf, x->st);
    x->bg = fwime_ctx::BgCache{};
    if (cudaMallocAsync(reinterpret_cast<void **>(&x->bg.buf), need, x->st) != cudaSuccess) {
        cudaGetLastError();
        x->bg.buf = nullptr;
        return false;
    }
    x->bg.bytes = need;
    return true;
}

// cache slot of state t (0: q^n0, 1: q^n0-1) of segment j for the batch starting at shot s0
static float *bg_slot(fwime_ctx *x, int j, int t, int s0)
{
    return x->bg.buf + ((2LL * j + t) * x->nshot + s0) * x->P;
}

// ---------------------------------------------------------------- gradient state (split gradient)
static size_t gs_bytes(const fwime_ctx *x, int K)
{
    const size_t nseg = (size_t)((x->g.nt - 1 + K - 1) / K);
    return (4 * nseg * (size_t)x->nshot * (size_t)x->P + (size_t)x->nshot * x->g.nt * x->nrec) * sizeof(float);
}

static void gs_release(fwime_ctx *x)
{
    if (x->gs.buf) cudaFreeAsync(x->gs.buf, x->st);
    x->gs = fwime_ctx::GradState{};
}

// Makes room for the state of every shot; false when it does not fit next to the adjoint sweep's own
// workspace for one shot (the split gradient then recomputes the forward sweep in its adjoint half).
static bool gs_reserve(fwime_ctx *x, int K)
{
    const size_t need = gs_bytes(x, K);
    if (x->gs.buf && x->gs.bytes >= need) return true;
    gs_release(x);
    const int nseg = (x->g.nt - 1 + K - 1) / K;
    const Sizes sz = op_sizes(x->g, x->nshot, x->nrec, x->P, x->NZ, x->NXP, FWIME_OP_GRADIENT, K, false, true);
    const size_t one = (sz.model + sz.per_shot) * sizeof(float) + ((size_t)2 << 30);
    (void)nseg;
    if (x->max_ws && x->ws_bytes + need + one > x->max_ws) return false;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (need + one > fr + x->ws_bytes) return false;
    if (cudaMallocAsync(reinterpret_cast<void **>(&x->gs.buf), need, x->st) != cudaSuccess) {
        cudaGetLastError();
        x->gs.buf = nullptr;
        return false;
    }
    x->gs.bytes = need;
    return true;
}

static int run_forward(fwime_ctx *x, Run &r, const float *v, const float *w, float *d)
{
    const int nt = x->g.nt, S = r.w.S;
    const size_t nd = (size_t)nt * x->nrec;
    for (int s0 = 0; s0 < x->nshot; s0 += S) {
        const int Sb = std::min(S, x->nshot - s0);
        float *cur = r.w.f[0], *prv = r.w.f[1];
        // both: the stencil never writes the inactive rows and columns, which must read as zero
        for (int i = 0; i < 2; ++i) TRY(zero(x, r.w.f[i], sizeof(float) * Sb * x->P));
        float *db = d + s0 * nd;
        TRY(zero(x, db, sizeof(float) * Sb * nd));
        // the launch of step n records its input q^n; the last sample q^{nt-1} is recorded after the loop
        for (int n = 0; n + 1 < nt; ++n) {
            TRY(prop(r, Sb, cur, prv, prv, nullptr, w + (size_t)s0 * nt + n, s0, nullptr, 0.f, nullptr, 0.f, nullptr,
                     0.f, nullptr, nullptr, RecTo{db + (size_t)n * x->nrec, 0}));
            std::swap(cur, prv);
        }
        TRY(record(r, Sb, cur, nullptr, db + (size_t)(nt - 1) * x->nrec, 0));
    }
    return FWIME_OK;
}

static int run_born(fwime_ctx *x, Run &r, const float *v, const float *w, const float *dv, float *d)
{
    const int nt = x->g.nt, S = r.w.S;
    const size_t nd = (size_t)nt * x->nrec;
    TRY(zero(x, r.w.coef, sizeof(float) * x->P));
    LAUNCH(FWIME_K_OTHER, 12.0 * x->g.nz * x->g.nx,
           launch_embed_scale(dv, r.w.bpad, r.w.coef, x->g.nz, x->g.nx, x->o, x->NXP, 1.f, x->st));
    for (int s0 = 0; s0 < x->nshot; s0 += S) {
        const int Sb = std::min(S, x->nshot - s0);
        float *c0 = r.w.f[0], *p0 = r.w.f[1], *c1 = r.w.f[2], *p1 = r.w.f[3], *D = r.w.f[4];
        for (int i = 0; i < 4; ++i) TRY(zero(x, r.w.f[i], sizeof(float) * Sb * x->P));
        float *db = d + s0 * nd;
        TRY(zero(x, db, sizeof(float) * Sb * nd));
        for (int n = 0; n + 1 < nt; ++n) {
            if (x->bg_written && n % r.w.K == 0) {
                TRY(copyf(x, bg_slot(x, n / r.w.K, 0, s0), c0, (size_t)Sb * x->P));
                TRY(copyf(x, bg_slot(x, n / r.w.K, 1, s0), p0, (size_t)Sb * x->P));
            }
            TRY(prop(r, Sb, c0, p0, p0, D, w + (size_t)s0 * nt + n, s0));
            TRY(prop(r, Sb, c1, p1, p1, nullptr, nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 0, r.w.coef, D,
                     RecTo{db + (size_t)n * x->nrec, 0}));
            std::swap(c0, p0);
            std::swap(c1, p1);
        }
        TRY(record(r, Sb, c1, nullptr, db + (size_t)(nt - 1) * x->nrec, 0));
    }
    return FWIME_OK;
}

static int run_born_ext(fwime_ctx *x, Run &r, const float *v, const float *w, const float *pt, float *d)
{
    const int nt = x->g.nt, S = r.w.S, K = r.w.K;
    const size_t nd = (size_t)nt * x->nrec;
    const long long SP = (long long)S * x->P;
    TRY(zero(x, r.w.W, sizeof(float) * x->g.nh * x->P));
    LAUNCH(FWIME_K_OTHER, 12.0 * x->g.nh * x->g.nz * x->g.nx,
           launch_ext_weights(pt, r.w.bpad, nullptr, nullptr, r.w.W, x->g.nh, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 0,
                              x->st));
    float *Dr = r.w.ring[0], *Er = r.w.ring[1];
    TRY(zero(x, Er, sizeof(float) * K * SP));
    for (int s0 = 0; s0 < x->nshot; s0 += S) {
        const int Sb = std::min(S, x->nshot - s0);
        float *c0 = r.w.f[0], *p0 = r.w.f[1], *c1 = r.w.f[2], *p1 = r.w.f[3];
        // all four: the stencil never writes the inactive rows and columns, which must read as zero
        for (int i = 0; i < 4; ++i) TRY(zero(x, r.w.f[i], sizeof(float) * Sb * x->P));
        float *db = d + s0 * nd;
        TRY(zero(x, db, sizeof(float) * Sb * nd));
        for (int n0 = 0; n0 < nt - 1; n0 += K) {
            const int n1 = std::min(n0 + K, nt - 1), kk = n1 - n0;
            if (x->bg_written) {
                TRY(copyf(x, bg_slot(x, n0 / K, 0, s0), c0, (size_t)Sb * x->P));
                TRY(copyf(x, bg_slot(x, n0 / K, 1, s0), p0, (size_t)Sb * x->P));
            }
            for (int n = n0; n < n1; ++n) {
                TRY(prop(r, Sb, c0, p0, p0, Dr + (n - n0) * SP, w + (size_t)s0 * nt + n, s0));
                std::swap(c0, p0);
            }
            TRY(scatter(r, Sb, n0, kk, r.w.W, ringref(Dr, SP, 0, 0), ringref(Er, SP, 0, 0), +1, 0));
            for (int n = n0; n < n1; ++n) {
                TRY(prop(r, Sb, c1, p1, p1, nullptr, nullptr, 0, Er + (n - n0) * SP, 1.f, nullptr, 0.f, nullptr, 0.f,
                         nullptr, nullptr, RecTo{db + (size_t)n * x->nrec, 0}));
                std::swap(c1, p1);
            }
        }
        TRY(record(r, Sb, c1, nullptr, db + (size_t)(nt - 1) * x->nrec, 0));
    }
    return FWIME_OK;
}

// B* (ext = false) and B~* (ext = true)
static int run_born_adj(fwime_ctx *x, Run &r, bool ext, const float *v, const float *w, const float *d, float *out,
                        int accumulate, bool use_bg)
{
    const int nt = x->g.nt, S = r.w.S, K = r.w.K, R = r.w.R, nseg = r.w.nseg;
    const size_t nd = (size_t)nt * x->nrec;
    const long long SP = (long long)S * x->P;
    const int planes = ext ? x->g.nh : 1;
    TRY(zero(x, r.w.acc1, sizeof(float) * planes * x->P));
    float *Dr = r.w.ring[0], *Mu = r.w.ring[1], *ck = r.w.ckpt;
    for (int s0 = 0; s0 < x->nshot; s0 += S) {
        const int Sb = std::min(S, x->nshot - s0);
        const size_t fb = sizeof(float) * (size_t)Sb * x->P;
        float *cur = r.w.f[0], *prv = r.w.f[1];
        // both: the stencil never writes the inactive rows and columns, which must read as zero
        for (int i = 0; i < 2; ++i) TRY(zero(x, r.w.f[i], fb));
        TRY(zero(x, Mu, sizeof(float) * R * SP));
        const float *ws = w + (size_t)s0 * nt;
        // checkpoint (q^{n0}, q^{n0-1}) at every segment start: from the background cache, or a forward sweep
        auto ckp = [&](int j, int t) -> float * { return use_bg ? bg_slot(x, j, t, s0) : ck + (2LL * j + t) * SP; };
        for (int j = 0; j < nseg && !use_bg; ++j) {
            TRY(copyf(x, ck + (2LL * j) * SP, cur, (size_t)Sb * x->P));
            TRY(copyf(x, ck + (2LL * j + 1) * SP, prv, (size_t)Sb * x->P));
            if (j == nseg - 1) break;
            for (int n = j * K; n < (j + 1) * K; ++n) {
                TRY(prop(r, Sb, cur, prv, prv, nullptr, ws + n, s0));
                std::swap(cur, prv);
            }
        }
        // backward sweep
        for (int j = nseg - 1; j >= 0; --j) {
            const int n0 = j * K, n1 = std::min(n0 + K, nt - 1), kk = n1 - n0;
            TRY(copyf(x, cur, ckp(j, 0), (size_t)Sb * x->P));
            TRY(copyf(x, prv, ckp(j, 1), (size_t)Sb * x->P));
            for (int n = n0; n < n1; ++n) {
                TRY(prop(r, Sb, cur, prv, prv, Dr + (n - n0) * SP, ws + n, s0));
                std::swap(cur, prv);
            }
            for (int m = n1; m >= n0 + 1; --m) {
                float *mo = Mu + (m % R) * SP;
                TRY(adj_step(r, Sb, Mu + ((m + 1) % R) * SP, Mu + ((m + 2) % R) * SP, mo, d + s0 * nd + (size_t)m * x->nrec));
            }
            if (ext)
                TRY(image(r, Sb, n0, kk, IMG_EXT, ringref(Dr, SP, 0, 0), ringref(Mu, SP, R, 1), ringref(nullptr, 0, 0, 0),
                          ringref(nullptr, 0, 0, 0), 1.f, nullptr, r.w.acc1));
            else
                TRY(image(r, Sb, n0, kk, IMG_LOCAL, ringref(Dr, SP, 0, 0), ringref(Mu, SP, R, 1),
                          ringref(nullptr, 0, 0, 0), ringref(nullptr, 0, 0, 0), 1.f, nullptr, r.w.acc1));
        }
    }
    LAUNCH(FWIME_K_OTHER, 12.0 * planes * x->g.nz * x->g.nx,
           launch_finalize(r.w.acc1, nullptr, r.w.bpad, v, out, planes, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 0,
                           accumulate, x->st));
    return FWIME_OK;
}

// ---------------------------------------------------------------- time-lag extension

static int tlag_launch(Run &r, int Sb, int n0, int n1, bool image, RingRef D, RingRef E, RingRef L, float *img,
                       const float *W = nullptr, int sigma = 1, int accumulate = 0)
{
    fwime_ctx *x = r.x;
    TlagArgs a{};
    a.NXP = x->NXP; a.nh = x->g.nh; a.S = Sb; a.lag = x->opt_tlag; a.nt = x->g.nt; a.n0 = n0; a.n1 = n1;
    a.jc = tlag_jc(r.w.K, x->opt_tlag, x->g.nh);
    a.P = x->P; a.sigma = sigma;
    a.z_lo = x->o; a.z_hi = x->o + x->g.nz; a.x_lo = x->o; a.x_hi = x->o + x->g.nx;
    a.W = W ? W : r.w.W; a.D = D; a.E = E; a.L = L; a.img = img; a.accumulate = accumulate;
    const double pts = (double)Sb * x->g.nz * x->g.nx * (n1 - n0);
    if (image) LAUNCH(FWIME_K_IMAGE, pts * 8.0 + 8.0 * x->g.nh * x->g.nz * x->g.nx, launch_tlag_image(a, x->st));
    else LAUNCH(FWIME_K_SCATTER, pts * 8.0 + 4.0 * x->g.nh * x->g.nz * x->g.nx, launch_tlag_scatter(a, x->st));
    return FWIME_OK;
}

// B~ with time lags: the background runs Hs = 2 hm lag steps ahead of the scattered field so that every
// segment's secondary sources find D2t q0 at n - 2 s_i for all lags in the ring
static int run_born_tlag(fwime_ctx *x, Run &r, const float *w, const float *pt, float *d)
{
    const int nt = x->g.nt, S = r.w.S, K = r.w.K, Hs = tlag_Hs(x->g, x->opt_tlag), RD = K + 2 * Hs;
    const size_t nd = (size_t)nt * x->nrec;
    const long long SP = (long long)S * x->P;
    TRY(zero(x, r.w.W, sizeof(float) * x->g.nh * x->P));
    LAUNCH(FWIME_K_OTHER, 12.0 * x->g.nh * x->g.nz * x->g.nx,
           launch_ext_weights(pt, r.w.bpad, nullptr, nullptr, r.w.W, x->g.nh, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 0,
                              x->st));
    float *Dr = r.w.ring[0], *Er = r.w.ring[1];
    TRY(zero(x, Er, sizeof(float) * K * SP));
    for (int s0 = 0; s0 < x->nshot; s0 += S) {
        const int Sb = std::min(S, x->nshot - s0);
        float *c0 = r.w.f[0], *p0 = r.w.f[1], *c1 = r.w.f[2], *p1 = r.w.f[3];
        for (int i = 0; i < 4; ++i) TRY(zero(x, r.w.f[i], sizeof(float) * Sb * x->P));
        float *db = d + s0 * nd;
        TRY(zero(x, db, sizeof(float) * Sb * nd));
        int bg = 0;   // next background step (produces D2t of that step)
        for (int n0 = 0; n0 < nt - 1; n0 += K) {
            const int n1 = std::min(n0 + K, nt - 1);
            for (const int top = std::min(n1 - 1 + Hs, nt - 2); bg <= top; ++bg) {
                TRY(prop(r, Sb, c0, p0, p0, Dr + (long long)(bg % RD) * SP, w + (size_t)s0 * nt + bg, s0));
                std::swap(c0, p0);
            }
            TRY(tlag_launch(r, Sb, n0, n1, false, ringref(Dr, SP, RD, 0), ringref(Er, SP, 0, 0),
                            ringref(nullptr, 0, 0, 0), nullptr));
            for (int n = n0; n < n1; ++n) {
                TRY(prop(r, Sb, c1, p1, p1, nullptr, nullptr, 0, Er + (n - n0) * SP, 1.f, nullptr, 0.f, nullptr, 0.f,
                         nullptr, nullptr, RecTo{db + (size_t)n * x->nrec, 0}));
                std::swap(c1, p1);
            }
        }
        TRY(record(r, Sb, c1, nullptr, db + (size_t)(nt - 1) * x->nrec, 0));
    }
    return FWIME_OK;
}

// B~* with time lags.  Output segments j = nseg-1 .. 0 need the background's D2t on [jK - Hs, (j+1)K - 1 + Hs];
// walking backwards, segment j adds the block [jK - Hs, (j+1)K - Hs), recomputed from the state stored at its
// start by a forward checkpointing sweep, so every D2t step is recomputed once.
static int run_born_tlag_adj(fwime_ctx *x, Run &r, const float *v, const float *w, const float *d, float *out,
                             int accumulate)
{
    const int nt = x->g.nt, S = r.w.S, K = r.w.K, R = r.w.R, nseg = r.w.nseg;
    const int Hs = tlag_Hs(x->g, x->opt_tlag), RD = K + 2 * Hs, NB = tlag_blocks(x->g, K, x->opt_tlag);
    const size_t nd = (size_t)nt * x->nrec;
    const long long SP = (long long)S * x->P;
    TRY(zero(x, r.w.acc1, sizeof(float) * x->g.nh * x->P));
    float *Dr = r.w.ring[0], *Mu = r.w.ring[1], *ck = r.w.ckpt;
    auto bstart = [&](int j) { return std::max(j * K - Hs, 0); };
    auto bend = [&](int j) { return std::min((j + 1) * K - Hs, nt - 1); };   // exclusive; D2t steps end at nt-2
    for (int s0 = 0; s0 < x->nshot; s0 += S) {
        const int Sb = std::min(S, x->nshot - s0);
        const size_t fb = sizeof(float) * (size_t)Sb * x->P;
        float *cur = r.w.f[0], *prv = r.w.f[1];
        TRY(zero(x, cur, fb));
        TRY(zero(x, prv, fb));
        TRY(zero(x, Mu, sizeof(float) * R * SP));
        const float *ws = w + (size_t)s0 * nt;
        // checkpointing sweep: the state at the start of every block
        int n = 0;
        for (int j = 0; j < NB; ++j) {
            const int b0 = bstart(j);
            if (b0 >= bend(j)) continue;   // empty block (all before step 0)
            for (; n < b0; ++n) {
                TRY(prop(r, Sb, cur, prv, prv, nullptr, ws + n, s0));
                std::swap(cur, prv);
            }
            TRY(copyf(x, ck + (2LL * j) * SP, cur, (size_t)Sb * x->P));
            TRY(copyf(x, ck + (2LL * j + 1) * SP, prv, (size_t)Sb * x->P));
        }
        auto block = [&](int j) -> int {   // recompute block j's D2t into the ring
            const int b0 = bstart(j), b1 = bend(j);
            if (b0 >= b1) return FWIME_OK;
            TRY(copyf(x, cur, ck + (2LL * j) * SP, (size_t)Sb * x->P));
            TRY(copyf(x, prv, ck + (2LL * j + 1) * SP, (size_t)Sb * x->P));
            for (int m = b0; m < b1; ++m) {
                TRY(prop(r, Sb, cur, prv, prv, Dr + (long long)(m % RD) * SP, ws + m, s0));
                std::swap(cur, prv);
            }
            return FWIME_OK;
        };
        int next_block = NB - 1;   // blocks > next_block are in the ring
        for (int j = nseg - 1; j >= 0; --j) {
            const int n0 = j * K, n1 = std::min(n0 + K, nt - 1);
            for (; next_block >= j; --next_block) TRY(block(next_block));
            for (int m = n1; m >= n0 + 1; --m) {
                float *mo = Mu + (m % R) * SP;
                TRY(adj_step(r, Sb, Mu + ((m + 1) % R) * SP, Mu + ((m + 2) % R) * SP, mo, d + s0 * nd + (size_t)m * x->nrec));
            }
            TRY(tlag_launch(r, Sb, n0, n1, true, ringref(Dr, SP, RD, 0), ringref(nullptr, 0, 0, 0),
                            ringref(Mu, SP, R, 1), r.w.acc1));
        }
    }
    LAUNCH(FWIME_K_OTHER, 12.0 * x->g.nh * x->g.nz * x->g.nx,
           launch_finalize(r.w.acc1, nullptr, r.w.bpad, v, out, x->g.nh, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 0,
                           accumulate, x->st));
    return FWIME_OK;
}

// T with time lags: the background q0 and the Born wavefield dq0 of dv run Hs steps ahead (their D2t in rings
// of K + 2 Hs steps), the extended Born wavefield dqs and the tomographic wavefield follow segment by segment
static int run_tomo_tlag(fwime_ctx *x, Run &r, const float *v, const float *w, const float *pt, const float *dv,
                         float *d)
{
    const int nt = x->g.nt, S = r.w.S, K = r.w.K, Hs = tlag_Hs(x->g, x->opt_tlag), RD = K + 2 * Hs;
    const size_t nd = (size_t)nt * x->nrec;
    const long long SP = (long long)S * x->P;
    const size_t nhP = (size_t)x->g.nh * x->P;
    TRY(zero(x, r.w.W, sizeof(float) * nhP));
    TRY(zero(x, r.w.W2, sizeof(float) * nhP));
    TRY(zero(x, r.w.coef, sizeof(float) * x->P));
    const double nm = (double)x->g.nz * x->g.nx;
    LAUNCH(FWIME_K_OTHER, 12.0 * x->g.nh * nm,
           launch_ext_weights(pt, r.w.bpad, nullptr, nullptr, r.w.W, x->g.nh, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 0,
                              x->st));
    LAUNCH(FWIME_K_OTHER, 20.0 * x->g.nh * nm,
           launch_ext_weights(pt, r.w.bpad, dv, v, r.w.W2, x->g.nh, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 1, x->st));
    LAUNCH(FWIME_K_OTHER, 12.0 * nm,
           launch_embed_scale(dv, r.w.bpad, r.w.coef, x->g.nz, x->g.nx, x->o, x->NXP, 1.f, x->st));
    float *D0r = r.w.ring[0], *Dq0r = r.w.ring[1], *Er = r.w.ring[2], *Dsr = r.w.ring[3];
    TRY(zero(x, Er, sizeof(float) * K * SP));
    const RingRef none = ringref(nullptr, 0, 0, 0), er = ringref(Er, SP, 0, 0);
    for (int s0 = 0; s0 < x->nshot; s0 += S) {
        const int Sb = std::min(S, x->nshot - s0);
        float *f[8];
        for (int i = 0; i < 8; ++i) {
            f[i] = r.w.f[i];
            TRY(zero(x, f[i], sizeof(float) * Sb * x->P));
        }
        float *db = d + s0 * nd;
        TRY(zero(x, db, sizeof(float) * Sb * nd));
        const float *ws = w + (size_t)s0 * nt;
        int bg = 0;
        for (int n0 = 0; n0 < nt - 1; n0 += K) {
            const int n1 = std::min(n0 + K, nt - 1);
            for (const int top = std::min(n1 - 1 + Hs, nt - 2); bg <= top; ++bg) {
                float *D0 = D0r + (long long)(bg % RD) * SP;
                TRY(prop(r, Sb, f[0], f[1], f[1], D0, ws + bg, s0));                       // background q0
                std::swap(f[0], f[1]);
                TRY(prop(r, Sb, f[2], f[3], f[3], Dq0r + (long long)(bg % RD) * SP, nullptr, 0, nullptr, 0, nullptr, 0,
                         nullptr, 0, r.w.coef, D0));                                            // Born wavefield of dv
                std::swap(f[2], f[3]);
            }
            TRY(tlag_launch(r, Sb, n0, n1, false, ringref(D0r, SP, RD, 0), er, none, nullptr));
            for (int n = n0; n < n1; ++n) {   // extended Born wavefield of p~
                TRY(prop(r, Sb, f[4], f[5], f[5], Dsr + (n - n0) * SP, nullptr, 0, Er + (n - n0) * SP, 1.f));
                std::swap(f[4], f[5]);
            }
            TRY(tlag_launch(r, Sb, n0, n1, false, ringref(D0r, SP, RD, 0), er, none, nullptr, r.w.W2, 1, 0));
            TRY(tlag_launch(r, Sb, n0, n1, false, ringref(Dq0r, SP, RD, 0), er, none, nullptr, r.w.W, 1, 1));
            for (int n = n0; n < n1; ++n) {   // tomographic wavefield
                TRY(prop(r, Sb, f[6], f[7], f[7], nullptr, nullptr, 0, Er + (n - n0) * SP, 1.f, nullptr, 0, nullptr, 0,
                         r.w.coef, Dsr + (n - n0) * SP, RecTo{db + (size_t)n * x->nrec, 0}));
                std::swap(f[6], f[7]);
            }
        }
        TRY(record(r, Sb, f[6], nullptr, db + (size_t)(nt - 1) * x->nrec, 0));
    }
    return FWIME_OK;
}

// T*, the FWIME gradient and the objective with time lags (modes as run_tomo_adj).  Forward sweep: q0 runs Hs
// steps ahead (its state stored at every block start), dqs follows segment by segment (its state stored at
// every segment start), both recorded for the residual.  Backward sweep: per segment, add the block of q0's
// D2t, recompute dqs, run the residual's adjoint field Hs steps ahead (the transposed lag scatter reads it
// up to Hs steps either way), then the second adjoint field and the images.
static int run_tomo_adj_tlag(fwime_ctx *x, Run &r, int mode, const float *v, const float *w, const float *pt,
                             const float *d, float *out, int accumulate, float eps)
{
    const bool grad = mode >= 1, objective_only = mode == 2;
    const int nt = x->g.nt, S = r.w.S, K = r.w.K, R = r.w.R, nseg = r.w.nseg;
    const int Hs = tlag_Hs(x->g, x->opt_tlag), RD = K + 2 * Hs, RM = RD + 2, NB = tlag_blocks(x->g, K, x->opt_tlag);
    const size_t nd = (size_t)nt * x->nrec;
    const long long SP = (long long)S * x->P;
    const size_t nhP = (size_t)x->g.nh * x->P;
    TRY(zero(x, r.w.W, sizeof(float) * nhP));
    TRY(zero(x, r.w.acc1, sizeof(float) * x->P));
    TRY(zero(x, r.w.acc2, sizeof(float) * nhP));
    const double nm = (double)x->g.nz * x->g.nx;
    LAUNCH(FWIME_K_OTHER, 12.0 * x->g.nh * nm,
           launch_ext_weights(pt, r.w.bpad, nullptr, nullptr, r.w.W, x->g.nh, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 0,
                              x->st));
    float *D0r = r.w.ring[0], *Er = r.w.ring[1], *Dsr = r.w.ring[2];
    float *Mu = r.w.ring[3], *Zr = r.w.ring[4], *Mu2 = r.w.ring[5];
    float *ckq = r.w.ckpt, *cks = r.w.ckpt + 2LL * NB * SP;
    TRY(zero(x, Er, sizeof(float) * K * SP));
    if (grad) TRY(zero(x, x->d_J, sizeof(double)));
    const int nred = 1024;
    const float idt2 = (float)(1.0 / ((double)x->g.dt * x->g.dt));
    const RingRef none = ringref(nullptr, 0, 0, 0), er = ringref(Er, SP, 0, 0), dring = ringref(D0r, SP, RD, 0);
    auto bstart = [&](int j) { return std::max(j * K - Hs, 0); };
    auto bend = [&](int j) { return std::min((j + 1) * K - Hs, nt - 1); };
    for (int s0 = 0; s0 < x->nshot; s0 += S) {
        const int Sb = std::min(S, x->nshot - s0);
        const size_t fb = sizeof(float) * (size_t)Sb * x->P;
        const size_t fn = (size_t)Sb * x->P;
        float *q0c = r.w.f[0], *q0p = r.w.f[1], *qsc = r.w.f[2], *qsp = r.w.f[3];
        for (int i = 0; i < 4; ++i) TRY(zero(x, r.w.f[i], fb));
        if (!objective_only) {
            TRY(zero(x, Mu, sizeof(float) * RM * SP));
            TRY(zero(x, Zr, sizeof(float) * R * SP));
            TRY(zero(x, Mu2, sizeof(float) * R * SP));
        }
        const float *ws = w + (size_t)s0 * nt;
        float *pred = r.w.pred;
        if (grad) TRY(zero(x, pred, sizeof(float) * Sb * nd));
        // forward sweep
        int bg = 0, nblk = 0;
        for (int j = 0; j < nseg; ++j) {
            const int n0 = j * K, n1 = std::min(n0 + K, nt - 1);
            if (!objective_only) {
                TRY(copyf(x, cks + (2LL * j) * SP, qsc, fn));
                TRY(copyf(x, cks + (2LL * j + 1) * SP, qsp, fn));
            }
            for (const int top = std::min(n1 - 1 + Hs, nt - 2); bg <= top; ++bg) {
                for (; !objective_only && nblk < NB && bstart(nblk) <= bg; ++nblk) {
                    if (bstart(nblk) < bend(nblk) && bstart(nblk) == bg) {
                        TRY(copyf(x, ckq + (2LL * nblk) * SP, q0c, fn));
                        TRY(copyf(x, ckq + (2LL * nblk + 1) * SP, q0p, fn));
                    }
                }
                TRY(prop(r, Sb, q0c, q0p, q0p, D0r + (long long)(bg % RD) * SP, ws + bg, s0));
                if (grad) TRY(record(r, Sb, q0p, nullptr, pred + (size_t)(bg + 1) * x->nrec, 0));
                std::swap(q0c, q0p);
            }
            TRY(tlag_launch(r, Sb, n0, n1, false, dring, er, none, nullptr));
            for (int n = n0; n < n1; ++n) {
                TRY(prop(r, Sb, qsc, qsp, qsp, nullptr, nullptr, 0, Er + (n - n0) * SP, 1.f));
                if (grad) TRY(record(r, Sb, qsp, nullptr, pred + (size_t)(n + 1) * x->nrec, 1));
                std::swap(qsc, qsp);
            }
        }
        const float *rr = d + s0 * nd;
        if (grad) {
            LAUNCH(FWIME_K_OTHER, 12.0 * Sb * nd,
                   launch_residual(pred, d + s0 * nd, pred, (long long)Sb * nd, x->d_part, nred, x->st));
            LAUNCH(FWIME_K_OTHER, 8.0 * nred, launch_sum_partials(x->d_part, nred, x->d_J, 1, 1.0, x->st));
            rr = pred;
        }
        if (objective_only) continue;
        // backward sweep
        int next_block = NB - 1, mu_lo = nt;   // mu^k computed for k >= mu_lo (mu^nt = mu^nt+1 = 0)
        for (int j = nseg - 1; j >= 0; --j) {
            const int n0 = j * K, n1 = std::min(n0 + K, nt - 1), kk = n1 - n0;
            for (; next_block >= j; --next_block) {   // q0's D2t block [b0, b1) from its checkpoint
                const int b0 = bstart(next_block), b1 = bend(next_block);
                if (b0 >= b1) continue;
                TRY(copyf(x, q0c, ckq + (2LL * next_block) * SP, fn));
                TRY(copyf(x, q0p, ckq + (2LL * next_block + 1) * SP, fn));
                for (int m = b0; m < b1; ++m) {
                    TRY(prop(r, Sb, q0c, q0p, q0p, D0r + (long long)(m % RD) * SP, ws + m, s0));
                    std::swap(q0c, q0p);
                }
            }
            TRY(copyf(x, qsc, cks + (2LL * j) * SP, fn));
            TRY(copyf(x, qsp, cks + (2LL * j + 1) * SP, fn));
            TRY(tlag_launch(r, Sb, n0, n1, false, dring, er, none, nullptr));
            for (int n = n0; n < n1; ++n) {
                TRY(prop(r, Sb, qsc, qsp, qsp, Dsr + (n - n0) * SP, nullptr, 0, Er + (n - n0) * SP, 1.f));
                std::swap(qsc, qsp);
            }
            // the residual's adjoint field, Hs steps ahead: mu^k down to k = n0 - Hs + 1
            for (const int lo = std::max(n0 - Hs + 1, 1); mu_lo - 1 >= lo; --mu_lo) {
                const int k = mu_lo - 1;
                float *mo = Mu + (long long)(k % RM) * SP;
                TRY(adj_step(r, Sb, Mu + (long long)((k + 1) % RM) * SP, Mu + (long long)((k + 2) % RM) * SP, mo,
                             rr + (size_t)k * x->nrec));
            }
            // z^m = sum_i W_i lambda^(m + 2 s_i) for m in [n0, n1) (lambda^n = mu^(n+1))
            TRY(tlag_launch(r, Sb, n0, n1, false, ringref(Mu, SP, RM, 1), ringref(Zr, SP, R, n0), none, nullptr, r.w.W,
                            -1, 0));
            // second adjoint field driven by d2t^T z
            for (int m = n1; m >= n0 + 1; --m) {
                TRY(prop(r, Sb, Mu2 + ((m + 1) % R) * SP, Mu2 + ((m + 2) % R) * SP, Mu2 + (m % R) * SP, nullptr,
                         nullptr, 0, Zr + ((m - 1) % R) * SP, idt2, Zr + (m % R) * SP, -2.f * idt2,
                         Zr + ((m + 1) % R) * SP, idt2));
            }
            TRY(image(r, Sb, n0, kk, IMG_LOCAL, dring, ringref(Mu, SP, RM, 1), ringref(Mu2, SP, R, 1),
                      ringref(Dsr, SP, 0, 0), grad ? 1.f : 0.f, nullptr, r.w.acc1));
            TRY(tlag_launch(r, Sb, n0, n1, true, dring, none, ringref(Mu, SP, RM, 1), r.w.acc2));
        }
    }
    if (!objective_only)
        LAUNCH(FWIME_K_OTHER, 20.0 * nm,
               launch_finalize(r.w.acc1, r.w.acc2, r.w.bpad, v, out, 1, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 1,
                               accumulate, x->st, pt, x->g.nh));
    if (grad) {
        LAUNCH(FWIME_K_OTHER, 4.0 * x->g.nh * nm,
               launch_dso(pt, x->g.nh, (long long)x->g.nz * x->g.nx, x->d_part, nred, x->st));
        LAUNCH(FWIME_K_OTHER, 8.0 * nred,
               launch_sum_partials(x->d_part, nred, x->d_J, 1, 0.5 * (double)eps * (double)eps, x->st));
        CK(cudaMemcpyAsync(x->h_J, x->d_J, sizeof(double), cudaMemcpyDeviceToHost, x->st));
    }
    return FWIME_OK;
}

static int run_tomo(fwime_ctx *x, Run &r, const float *v, const float *w, const float *pt, const float *dv, float *d)
{
    const int nt = x->g.nt, S = r.w.S, K = r.w.K;
    const size_t nd = (size_t)nt * x->nrec;
    const long long SP = (long long)S * x->P;
    const size_t nhP = (size_t)x->g.nh * x->P;
    TRY(zero(x, r.w.W, sizeof(float) * nhP));
    TRY(zero(x, r.w.W2, sizeof(float) * nhP));
    TRY(zero(x, r.w.coef, sizeof(float) * x->P));
    const double nm = (double)x->g.nz * x->g.nx;
    LAUNCH(FWIME_K_OTHER, 12.0 * x->g.nh * nm,
           launch_ext_weights(pt, r.w.bpad, nullptr, nullptr, r.w.W, x->g.nh, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 0,
                              x->st));
    LAUNCH(FWIME_K_OTHER, 20.0 * x->g.nh * nm,
           launch_ext_weights(pt, r.w.bpad, dv, v, r.w.W2, x->g.nh, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 1, x->st));
    LAUNCH(FWIME_K_OTHER, 12.0 * nm,
           launch_embed_scale(dv, r.w.bpad, r.w.coef, x->g.nz, x->g.nx, x->o, x->NXP, 1.f, x->st));
    float *D0r = r.w.ring[0], *D0d = r.w.ring[1], *Er = r.w.ring[2], *Dsr = r.w.ring[3];
    TRY(zero(x, Er, sizeof(float) * K * SP));
    for (int s0 = 0; s0 < x->nshot; s0 += S) {
        const int Sb = std::min(S, x->nshot - s0);
        float *f[8];
        for (int i = 0; i < 8; ++i) {
            f[i] = r.w.f[i];
            TRY(zero(x, f[i], sizeof(float) * Sb * x->P));
        }
        float *db = d + s0 * nd;
        TRY(zero(x, db, sizeof(float) * Sb * nd));
        const float *ws = w + (size_t)s0 * nt;
        for (int n0 = 0; n0 < nt - 1; n0 += K) {
            const int n1 = std::min(n0 + K, nt - 1), kk = n1 - n0;
            for (int n = n0; n < n1; ++n) {   // background q0
                TRY(prop(r, Sb, f[0], f[1], f[1], D0r + (n - n0) * SP, ws + n, s0));
                std::swap(f[0], f[1]);
            }
            for (int n = n0; n < n1; ++n) {   // Born wavefield of dv
                TRY(prop(r, Sb, f[2], f[3], f[3], D0d + (n - n0) * SP, nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 0,
                         r.w.coef, D0r + (n - n0) * SP));
                std::swap(f[2], f[3]);
            }
            TRY(scatter(r, Sb, n0, kk, r.w.W, ringref(D0r, SP, 0, 0), ringref(Er, SP, 0, 0), +1, 0));
            for (int n = n0; n < n1; ++n) {   // extended Born wavefield of p~
                TRY(prop(r, Sb, f[4], f[5], f[5], Dsr + (n - n0) * SP, nullptr, 0, Er + (n - n0) * SP, 1.f));
                std::swap(f[4], f[5]);
            }
            TRY(scatter(r, Sb, n0, kk, r.w.W2, ringref(D0r, SP, 0, 0), ringref(Er, SP, 0, 0), +1, 0));
            TRY(scatter(r, Sb, n0, kk, r.w.W, ringref(D0d, SP, 0, 0), ringref(Er, SP, 0, 0), +1, 1));
            for (int n = n0; n < n1; ++n) {   // tomographic wavefield
                TRY(prop(r, Sb, f[6], f[7], f[7], nullptr, nullptr, 0, Er + (n - n0) * SP, 1.f, nullptr, 0, nullptr, 0,
                         r.w.coef, Dsr + (n - n0) * SP, RecTo{db + (size_t)n * x->nrec, 0}));
                std::swap(f[6], f[7]);
            }
        }
        TRY(record(r, Sb, f[6], nullptr, db + (size_t)(nt - 1) * x->nrec, 0));
    }
    return FWIME_OK;
}

// Phases of the FWIME gradient: both sweeps per batch (the self-contained call), the forward sweep alone
// leaving its checkpoints and residual in the context's gradient state, or the adjoint sweep alone from it.
enum { PH_BOTH = 0, PH_FORWARD = 1, PH_BACKWARD = 2 };

// T* (mode 0, r = d), the FWIME gradient (mode 1, r = f + B~p~ - dobs) and the
// objective alone (mode 2: forward sweep and residual norm, no adjoint sweep).
// With mode 1, `phase` splits the gradient into its forward sweep (checkpoints of the background and
// scattered fields of every shot at every segment start, and the residual, written to x->gs) and its
// adjoint sweep (read back from x->gs); PH_BOTH keeps both per batch in the workspace.
static int run_tomo_adj(fwime_ctx *x, Run &r, int mode, const float *v, const float *w, const float *pt,
                        const float *d, float *out, int accumulate, float eps, int phase = PH_BOTH)
{
    const bool grad = mode >= 1, objective_only = mode == 2 || phase == PH_FORWARD;
    const bool fwd = phase != PH_BACKWARD, bwd = !objective_only;
    const bool state = phase != PH_BOTH;   // checkpoints and residual in x->gs
    const int nt = x->g.nt, S = r.w.S, K = r.w.K, R = r.w.R, nseg = r.w.nseg;
    const size_t nd = (size_t)nt * x->nrec;
    const long long SP = (long long)S * x->P;
    const size_t nhP = (size_t)x->g.nh * x->P;
    TRY(zero(x, r.w.W, sizeof(float) * nhP));
    if (bwd) {
        TRY(zero(x, r.w.acc1, sizeof(float) * x->P));
        TRY(zero(x, r.w.acc2, sizeof(float) * nhP));   // extended image of the residual, contracted with p~ at the end
    }
    const double nm = (double)x->g.nz * x->g.nx;
    LAUNCH(FWIME_K_OTHER, 12.0 * x->g.nh * nm,
           launch_ext_weights(pt, r.w.bpad, nullptr, nullptr, r.w.W, x->g.nh, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 0,
                              x->st));
    float *D0r = r.w.ring[0], *Er = r.w.ring[1], *Dsr = r.w.ring[2];
    float *Mu = r.w.ring[3], *Zr = r.w.ring[4], *Mu2 = r.w.ring[5];
    float *ck = r.w.ckpt;
    TRY(zero(x, Er, sizeof(float) * K * SP));
    const bool report_J = grad && fwd;
    if (report_J) TRY(zero(x, x->d_J, sizeof(double)));
    const int nred = 1024;
    float *res_state = state ? x->gs.buf + 4LL * nseg * x->nshot * x->P : nullptr;
    for (int s0 = 0; s0 < x->nshot; s0 += S) {
        const int Sb = std::min(S, x->nshot - s0);
        const size_t fb = sizeof(float) * (size_t)Sb * x->P;
        const size_t fn = (size_t)Sb * x->P;
        // checkpoint t (0, 1: q0^n0, q0^n0-1; 2, 3: the scattered field's) of segment j for this batch
        auto ckp = [&](int j, int t) -> float * {
            return state ? x->gs.buf + ((4LL * j + t) * x->nshot + s0) * x->P : ck + (4LL * j + t) * SP;
        };
        float *q0c = r.w.f[0], *q0p = r.w.f[1], *qsc = r.w.f[2], *qsp = r.w.f[3];
        for (int i = 0; i < 4; ++i) TRY(zero(x, r.w.f[i], fb));
        if (bwd) {
            TRY(zero(x, Mu, sizeof(float) * R * SP));
            TRY(zero(x, Zr, sizeof(float) * R * SP));
            TRY(zero(x, Mu2, sizeof(float) * R * SP));
        }
        const float *ws = w + (size_t)s0 * nt;
        float *pred = state ? res_state + s0 * nd : r.w.pred;
        const float *rr = d + s0 * nd;
        if (fwd) {
            const bool keep = bwd || state;   // checkpoints for an adjoint sweep
            if (grad) TRY(zero(x, pred, sizeof(float) * Sb * nd));
            // forward sweep
            for (int j = 0; j < nseg; ++j) {
                if (keep) {
                    TRY(copyf(x, ckp(j, 0), q0c, fn));
                    TRY(copyf(x, ckp(j, 1), q0p, fn));
                    TRY(copyf(x, ckp(j, 2), qsc, fn));
                    TRY(copyf(x, ckp(j, 3), qsp, fn));
                }
                if (!grad && j == nseg - 1) break;
                const int n0 = j * K, n1 = std::min(n0 + K, nt - 1), kk = n1 - n0;
                // with the gradient, the launch of step n adds its input (q0^n, then the scattered field's)
                // to the prediction's row n (zeroed above; a + b is exact in either order of the two)
                for (int n = n0; n < n1; ++n) {
                    TRY(prop(r, Sb, q0c, q0p, q0p, D0r + (n - n0) * SP, ws + n, s0, nullptr, 0.f, nullptr, 0.f,
                             nullptr, 0.f, nullptr, nullptr, RecTo{grad ? pred + (size_t)n * x->nrec : nullptr, 1}));
                    std::swap(q0c, q0p);
                }
                TRY(scatter(r, Sb, n0, kk, r.w.W, ringref(D0r, SP, 0, 0), ringref(Er, SP, 0, 0), +1, 0));
                for (int n = n0; n < n1; ++n) {
                    TRY(prop(r, Sb, qsc, qsp, qsp, nullptr, nullptr, 0, Er + (n - n0) * SP, 1.f, nullptr, 0.f, nullptr,
                             0.f, nullptr, nullptr, RecTo{grad ? pred + (size_t)n * x->nrec : nullptr, 1}));
                    std::swap(qsc, qsp);
                }
            }
            if (grad) {   // the last sample of both fields
                TRY(record(r, Sb, q0c, qsc, pred + (size_t)(nt - 1) * x->nrec, 1));
                LAUNCH(FWIME_K_OTHER, 12.0 * Sb * nd,
                       launch_residual(pred, d + s0 * nd, pred, (long long)Sb * nd, x->d_part, nred, x->st));
                LAUNCH(FWIME_K_OTHER, 8.0 * nred, launch_sum_partials(x->d_part, nred, x->d_J, 1, 1.0, x->st));
            }
        }
        if (grad) rr = pred;
        if (!bwd) continue;
        // backward sweep
        for (int j = nseg - 1; j >= 0; --j) {
            const int n0 = j * K, n1 = std::min(n0 + K, nt - 1), kk = n1 - n0;
            TRY(copyf(x, q0c, ckp(j, 0), fn));
            TRY(copyf(x, q0p, ckp(j, 1), fn));
            TRY(copyf(x, qsc, ckp(j, 2), fn));
            TRY(copyf(x, qsp, ckp(j, 3), fn));
            for (int n = n0; n < n1; ++n) {
                TRY(prop(r, Sb, q0c, q0p, q0p, D0r + (n - n0) * SP, ws + n, s0));
                std::swap(q0c, q0p);
            }
            TRY(scatter(r, Sb, n0, kk, r.w.W, ringref(D0r, SP, 0, 0), ringref(Er, SP, 0, 0), +1, 0));
            for (int n = n0; n < n1; ++n) {
                TRY(prop(r, Sb, qsc, qsp, qsp, Dsr + (n - n0) * SP, nullptr, 0, Er + (n - n0) * SP, 1.f));
                std::swap(qsc, qsp);
            }
            // adjoint of the residual: mu^m, m = n1 .. n0+1 (lambda^ at step n is mu^{n+1}), each step also
            // writing its D2t, (mu^m - 2 mu^{m+1} + mu^{m+2}) / dt^2, at slot m - n0 - 1 of Zr
            for (int m = n1; m >= n0 + 1; --m) {
                float *mo = Mu + (m % R) * SP;
                TRY(adj_step(r, Sb, Mu + ((m + 1) % R) * SP, Mu + ((m + 2) % R) * SP, mo, rr + (size_t)m * x->nrec,
                             Zr + (m - n0 - 1) * SP));
            }
            // The second adjoint field's source d2t^T z, z^n = E_D^T(W, lambda^n): E_D^T acts on space only,
            // so y^m = (z^{m-1} - 2 z^m + z^{m+1}) / dt^2 = E_D^T(W, D2t of the step producing mu^m): one
            // transposed scatter of those D2t into slots m - n0 - 1 of the scattered-field ring (free again
            // once the recomputed q_s is past this segment; zero outside the scatter's columns, which only
            // scatters write)
            TRY(scatter(r, Sb, n0, kk, r.w.W, ringref(Zr, SP, 0, 0), ringref(Er, SP, 0, 0), -1, 0));
            for (int m = n1; m >= n0 + 1; --m) {
                TRY(prop(r, Sb, Mu2 + ((m + 1) % R) * SP, Mu2 + ((m + 2) % R) * SP, Mu2 + (m % R) * SP, nullptr,
                         nullptr, 0, Er + (m - n0 - 1) * SP, 1.f));
            }
            // the extended image of the residual's adjoint field (contracted with p~ at the end) and, in the
            // same launch, the local terms D0 (alpha lambda^ + mu2) + Ds lambda^
            TRY(image(r, Sb, n0, kk, IMG_EXT, ringref(D0r, SP, 0, 0), ringref(Mu, SP, R, 1), ringref(Mu2, SP, R, 1),
                      ringref(Dsr, SP, 0, 0), grad ? 1.f : 0.f, nullptr, r.w.acc2, r.w.acc1));
        }
    }
    if (bwd)
        LAUNCH(FWIME_K_OTHER, 20.0 * nm,
               launch_finalize(r.w.acc1, r.w.acc2, r.w.bpad, v, out, 1, x->g.nz, x->g.nx, x->o, x->NXP, x->P, 1,
                               accumulate, x->st, pt, x->g.nh));
    if (report_J) {
        LAUNCH(FWIME_K_OTHER, 4.0 * x->g.nh * nm,
               launch_dso(pt, x->g.nh, (long long)x->g.nz * x->g.nx, x->d_part, nred, x->st));
        LAUNCH(FWIME_K_OTHER, 8.0 * nred,
               launch_sum_partials(x->d_part, nred, x->d_J, 1, 0.5 * (double)eps * (double)eps, x->st));
        CK(cudaMemcpyAsync(x->h_J, x->d_J, sizeof(double), cudaMemcpyDeviceToHost, x->st));
    }
    return FWIME_OK;
}

// ----------------------------------------------------------- dispatch

struct Call {
    int op;
    const float *v, *w, *in1, *in2;
    float *out;
    int accumulate;
    float eps;
};

// internal operators of the split gradient (never passed through the C ABI)
enum { OP_GRAD_FWD = 100, OP_GRAD_BWD = 101 };

static bool is_bg_writer(int op) { return op == FWIME_OP_BORN || op == FWIME_OP_BORN_EXT; }
static bool is_bg_reader(int op) { return op == FWIME_OP_BORN_ADJ || op == FWIME_OP_BORN_EXT_ADJ; }
// the time-lag schedules place their checkpoints differently: no background cache for them
static bool bg_applies(const fwime_ctx *x, int op) { return !(x->opt_tlag > 0 && (op == FWIME_OP_BORN_EXT || op == FWIME_OP_BORN_EXT_ADJ)); }

// does this call start from the cached background checkpoints?
static bool bg_usable(const fwime_ctx *x, const Call &c)
{
    return is_bg_reader(c.op) && bg_applies(x, c.op) && x->opt_reuse_bg && x->bg.valid && x->bg.v == c.v &&
           x->bg.w == c.w && x->bg.K == seg_K(x) && x->bg.buf;
}

// host-side bookkeeping once a call has been enqueued (directly or as a graph replay)
static void bg_after(fwime_ctx *x, const Call &c, bool wrote)
{
    if (is_bg_writer(c.op)) {
        x->bg.valid = wrote && bg_applies(x, c.op);
        x->bg.v = c.v; x->bg.w = c.w; x->bg.K = seg_K(x);
    } else if (!is_bg_reader(c.op)) {
        x->bg.valid = false;
    }
}

static int enqueue(fwime_ctx *x, const Call &c)
{
    Run r;
    const bool use_bg = bg_usable(x, c);
    x->bg_used = use_bg;
    x->bg_written = is_bg_writer(c.op) && bg_applies(x, c.op) && x->opt_reuse_bg && bg_reserve(x, seg_K(x));
    if (x->bg_written) x->bg.valid = false;   // being overwritten
    if (c.op == OP_GRAD_FWD || c.op == OP_GRAD_BWD) {
        // the split gradient: checkpoints and residual live in the context's gradient state
        TRY(plan(x, c.op == OP_GRAD_FWD ? FWIME_OP_OBJECTIVE : FWIME_OP_GRADIENT, r.w, true));
        init_run(x, r, r.w.S);
        TRY(prep_model(x, r, c.v));
        return run_tomo_adj(x, r, 1, c.v, c.w, c.in1, c.in2, c.out, c.accumulate, c.eps,
                            c.op == OP_GRAD_FWD ? PH_FORWARD : PH_BACKWARD);
    }
    TRY(plan(x, c.op, r.w, use_bg));
    init_run(x, r, r.w.S);
    TRY(prep_model(x, r, c.v));
    switch (c.op) {
    case FWIME_OP_FORWARD: return run_forward(x, r, c.v, c.w, c.out);
    case FWIME_OP_BORN: return run_born(x, r, c.v, c.w, c.in1, c.out);
    case FWIME_OP_BORN_ADJ: return run_born_adj(x, r, false, c.v, c.w, c.in1, c.out, c.accumulate, use_bg);
    case FWIME_OP_BORN_EXT:
        if (x->opt_tlag > 0) return run_born_tlag(x, r, c.w, c.in1, c.out);
        return run_born_ext(x, r, c.v, c.w, c.in1, c.out);
    case FWIME_OP_BORN_EXT_ADJ:
        if (x->opt_tlag > 0) return run_born_tlag_adj(x, r, c.v, c.w, c.in1, c.out, c.accumulate);
        return run_born_adj(x, r, true, c.v, c.w, c.in1, c.out, c.accumulate, use_bg);
    case FWIME_OP_TOMO:
        if (x->opt_tlag > 0) return run_tomo_tlag(x, r, c.v, c.w, c.in1, c.in2, c.out);
        return run_tomo(x, r, c.v, c.w, c.in1, c.in2, c.out);
    case FWIME_OP_TOMO_ADJ:
    case FWIME_OP_GRADIENT:
    case FWIME_OP_OBJECTIVE: {
        const int mode = c.op == FWIME_OP_TOMO_ADJ ? 0 : (c.op == FWIME_OP_GRADIENT ? 1 : 2);
        float *o = c.op == FWIME_OP_OBJECTIVE ? nullptr : c.out;
        const int acc = c.op == FWIME_OP_OBJECTIVE ? 0 : c.accumulate;
        const float e = c.op == FWIME_OP_TOMO_ADJ ? 0.f : c.eps;
        if (x->opt_tlag > 0) return run_tomo_adj_tlag(x, r, mode, c.v, c.w, c.in1, c.in2, o, acc, e);
        return run_tomo_adj(x, r, mode, c.v, c.w, c.in1, c.in2, o, acc, e);
    }
    }
    return fail(x, FWIME_EINVAL, "unknown operator %d", c.op);
}

static int enqueue_noted(fwime_ctx *x, const Call &c)
{
    const int rc = enqueue(x, c);
    if (rc == FWIME_OK) bg_after(x, c, x->bg_written);
    return rc;
}

static int run_call(fwime_ctx *x, const Call &c)
{
    if (!x->opt_graph || x->opt_plain || x->opt_profile) {
        x->launches = 0;
        return enqueue_noted(x, c);
    }
    if (x->st == nullptr) return fail(x, FWIME_EINVAL, "graph mode needs a non-default stream");
    // plan (and reserve the background cache) first so that no allocation happens inside a capture
    const bool use_bg = bg_usable(x, c);
    const bool write_bg = is_bg_writer(c.op) && bg_applies(x, c.op) && x->opt_reuse_bg && bg_reserve(x, seg_K(x));
    {
        WS w;
        TRY(plan(x, c.op, w, use_bg));
    }
    char key[320];
    snprintf(key, sizeof(key), "%d|%p|%p|%p|%p|%p|%d|%a|%d|%d|%d|%d%d|%p|%d", c.op, (const void *)c.v, (const void *)c.w,
             (const void *)c.in1, (const void *)c.in2, (void *)c.out, c.accumulate, (double)c.eps, x->opt_S, x->opt_K,
             x->opt_zchunk, use_bg ? 1 : 0, write_bg ? 1 : 0, (const void *)(use_bg || write_bg ? x->bg.buf : nullptr),
             x->opt_tlag * 2 + x->opt_fs);
    auto it = x->graphs.find(key);
    if (it == x->graphs.end()) {
        CK(cudaStreamBeginCapture(x->st, cudaStreamCaptureModeThreadLocal));
        x->capturing = true;
        x->launches = 0;
        int rc = enqueue(x, c);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(x->st, &graph);
        x->capturing = false;
        if (rc != FWIME_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        CK(e);
        Graph gr;
        gr.launches = x->launches;
        e = cudaGraphInstantiate(&gr.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
        it = x->graphs.emplace(key, gr).first;
    }
    x->launches = it->second.launches;
    CK(cudaGraphLaunch(it->second.exec, x->st));
    x->bg_used = use_bg;
    bg_after(x, c, write_bg);
    return FWIME_OK;
}

// host-I/O wrapper: stage inputs, run, copy outputs back, wait
enum { K_NONE = 0, K_DATA, K_MODEL, K_EXT };

static int call_op(fwime_ctx *x, Call c, int kin1, int kin2, int kout)
{
    if (!x) return FWIME_EINVAL;
    NOT_SERVER(x);
    if (!c.v || !c.w || (!c.out && c.op != FWIME_OP_OBJECTIVE)) return fail(x, FWIME_EINVAL, "null pointer argument");
    if (!x->opt_host_io) return run_call(x, c);
    // the staged v and w sit at the start of the arena: a B~* can reuse the background of the B~ before it
    // (FWIME_OPT_REUSE_BACKGROUND) when the arena has not moved in between
    auto staged = [&](Call s) {
        s.v = reinterpret_cast<const float *>(x->ws);
        s.w = reinterpret_cast<const float *>(x->ws) + al((size_t)x->g.nz * x->g.nx);
        return s;
    };
    bool use_bg = x->ws && bg_usable(x, staged(c));
    WS w;
    TRY(plan(x, c.op, w, use_bg));
    if (use_bg && !bg_usable(x, staged(c))) TRY(plan(x, c.op, w, false));   // the arena moved
    const size_t nm = (size_t)x->g.nz * x->g.nx, nd = (size_t)x->nshot * x->g.nt * x->nrec;
    auto count = [&](int k) -> size_t {
        return k == K_DATA ? nd : (k == K_MODEL ? nm : (k == K_EXT ? (size_t)x->g.nh * nm : 0));
    };
    // staging: data in -> sd1, dv -> sdv, p~ -> sm1, data out -> sd2, model/image out -> smo
    auto stage_in = [&](int k) -> float * { return k == K_DATA ? w.sd1 : (k == K_MODEL ? w.sdv : w.sm1); };
    float *in1 = kin1 ? stage_in(kin1) : nullptr;
    float *in2 = kin2 ? stage_in(kin2) : nullptr;
    float *out = kout == K_DATA ? w.sd2 : (kout == K_NONE ? nullptr : w.smo);
    CK(cudaMemcpyAsync(w.sv, c.v, nm * sizeof(float), cudaMemcpyHostToDevice, x->st));
    CK(cudaMemcpyAsync(w.sw, c.w, (size_t)x->nshot * x->g.nt * sizeof(float), cudaMemcpyHostToDevice, x->st));
    if (in1) CK(cudaMemcpyAsync(in1, c.in1, count(kin1) * sizeof(float), cudaMemcpyHostToDevice, x->st));
    if (in2) CK(cudaMemcpyAsync(in2, c.in2, count(kin2) * sizeof(float), cudaMemcpyHostToDevice, x->st));
    if (c.accumulate) CK(cudaMemcpyAsync(out, c.out, count(kout) * sizeof(float), cudaMemcpyHostToDevice, x->st));
    float *user_out = c.out;
    c.v = w.sv; c.w = w.sw; c.in1 = in1; c.in2 = in2; c.out = out;
    x->launches = 0;
    TRY(enqueue_noted(x, c));
    if (kout != K_NONE) CK(cudaMemcpyAsync(user_out, out, count(kout) * sizeof(float), cudaMemcpyDeviceToHost, x->st));
    return fwime_sync(x);
}

// ================================================================ C ABI

extern "C" {

const char *fwime_strerror(int code)
{
    switch (code) {
    case FWIME_OK: return "ok";
    case FWIME_EINVAL: return "invalid argument";
    case FWIME_ENOMEM: return "out of device memory or over the workspace budget";
    case FWIME_ECFL: return "CFL condition violated or non-positive velocity";
    case FWIME_ECUDA: return "CUDA runtime error";
    case FWIME_ETIMEOUT: return "device-side wait timed out";
    case FWIME_EBUSY: return "context busy";
    }
    return "unknown error";
}

int fwime_workspace_bytes(const fwime_grid *g, const fwime_geom *geo, int op, int shots_per_batch, int segment,
                          size_t *bytes)
{
    if (validate(g, geo, nullptr) != FWIME_OK || !bytes || op < 0 || op > FWIME_OP_OBJECTIVE) return FWIME_EINVAL;
    const int NZ = g->nz + 2 * (g->sponge + 4), NX = g->nx + 2 * (g->sponge + 4), NXP = (NX + 31) / 32 * 32;
    const long long P = (long long)NZ * NXP;
    int K = segment > 0 ? segment : auto_K(g->nt);
    K = std::max(1, std::min(K, g->nt - 1));
    Sizes s = op_sizes(*g, geo->nshot, geo->nrec, P, NZ, NXP, op, K, false);
    const int S = shots_per_batch > 0 ? std::min(shots_per_batch, geo->nshot) : geo->nshot;
    *bytes = (s.model + s.per_shot * (size_t)S) * sizeof(float) + 4096;
    return FWIME_OK;
}

int fwime_create(fwime_ctx **out, const fwime_grid *g, const fwime_geom *geo, size_t max_workspace_bytes,
                 void *cuda_stream)
{
    if (!out) return FWIME_EINVAL;
    *out = nullptr;
    if (validate(g, geo, nullptr) != FWIME_OK) return FWIME_EINVAL;
    fwime_ctx *x = new fwime_ctx();
    x->g = *g;
    x->nshot = geo->nshot;
    x->nrec = geo->nrec;
    x->src_iz.assign(geo->src_iz, geo->src_iz + geo->nshot);
    x->src_ix.assign(geo->src_ix, geo->src_ix + geo->nshot);
    x->rec_iz.assign(geo->rec_iz, geo->rec_iz + geo->nrec);
    x->rec_ix.assign(geo->rec_ix, geo->rec_ix + geo->nrec);
    x->o = g->sponge + 4;
    x->NZ = g->nz + 2 * x->o;
    x->NX = g->nx + 2 * x->o;
    x->NXP = (x->NX + 31) / 32 * 32;
    x->P = (long long)x->NZ * x->NXP;
    x->st = reinterpret_cast<cudaStream_t>(cuda_stream);
    x->max_ws = max_workspace_bytes;
    cudaGetDevice(&x->device);
    // offsets: [src_off(nshot)][rec_off(nrec)]
    x->h_off.resize(x->nshot + x->nrec);
    for (int s = 0; s < x->nshot; ++s) x->h_off[s] = (x->src_iz[s] + x->o) * x->NXP + x->src_ix[s] + x->o;
    for (int r = 0; r < x->nrec; ++r)
        x->h_off[x->nshot + r] = (x->rec_iz[r] + x->o) * x->NXP + x->rec_ix[r] + x->o;
    // injection map: rows of the receivers x NXP (first receiver at a point, -1 elsewhere), then the chain
    int rlo = x->NZ, rhi = 0;
    for (int r = 0; r < x->nrec; ++r) {
        rlo = std::min(rlo, x->rec_iz[r] + x->o);
        rhi = std::max(rhi, x->rec_iz[r] + x->o + 1);
    }
    x->inj_lo = rlo;
    x->inj_hi = rhi;
    const size_t nmap = (size_t)(rhi - rlo) * x->NXP;
    x->h_inj.assign(nmap + x->nrec, -1);
    {
        std::vector<int> last(nmap, -1);
        for (int r = 0; r < x->nrec; ++r) {
            const size_t pos = (size_t)(x->rec_iz[r] + x->o - rlo) * x->NXP + x->rec_ix[r] + x->o;
            if (x->h_inj[pos] < 0) x->h_inj[pos] = r;
            else x->h_inj[nmap + last[pos]] = r;
            last[pos] = r;
        }
    }
    const size_t off_inj = ((1 + 1024) * sizeof(double) + sizeof(int) * (1 + x->h_off.size()) + 15) / 16 * 16;
    const size_t small_bytes = off_inj + sizeof(int) * x->h_inj.size();
    double *slot = pinned_slot();
    bool ok = slot != nullptr &&
              cudaMallocAsync(&x->small, small_bytes, x->st) == cudaSuccess;
    if (ok) {
        x->h_J = slot;
        x->h_status = reinterpret_cast<int *>(slot + 1);
        x->d_J = reinterpret_cast<double *>(x->small);
        x->d_part = x->d_J + 1;
        x->d_status = reinterpret_cast<int *>(x->d_part + 1024);
        x->d_src_off = x->d_status + 1;
        x->d_rec_off = x->d_src_off + x->nshot;
        x->d_inj_map = reinterpret_cast<int *>(reinterpret_cast<char *>(x->small) + off_inj);
        x->d_inj_next = x->d_inj_map + nmap;
        ok = cudaMemsetAsync(x->small, 0, small_bytes, x->st) == cudaSuccess &&
             cudaMemcpyAsync(x->d_src_off, x->h_off.data(), x->h_off.size() * sizeof(int), cudaMemcpyHostToDevice,
                             x->st) == cudaSuccess &&
             cudaMemcpyAsync(x->d_inj_map, x->h_inj.data(), x->h_inj.size() * sizeof(int), cudaMemcpyHostToDevice,
                             x->st) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        fwime_destroy(x);
        return FWIME_ENOMEM;
    }
    *x->h_J = 0.0;
    *out = x;
    return FWIME_OK;
}

void fwime_destroy(fwime_ctx *x)
{
    if (!x) return;
    if (x->srv) {
        server_destroy(x->srv);
        delete x;
        return;
    }
    if (x->st) cudaStreamSynchronize(x->st);
    else cudaDeviceSynchronize();
    for (auto &kv : x->graphs) cudaGraphExecDestroy(kv.second.exec);
    for (auto e : x->ev) cudaEventDestroy(e);
    if (x->ws) cudaFreeAsync(x->ws, x->st);
    if (x->small) cudaFreeAsync(x->small, x->st);
    if (x->vp_hist_dev) cudaFreeAsync(x->vp_hist_dev, x->st);
    if (x->bg.buf) cudaFreeAsync(x->bg.buf, x->st);
    if (x->gs.buf) cudaFreeAsync(x->gs.buf, x->st);
    cudaGetLastError();
    delete x;
}

int fwime_set_option(fwime_ctx *x, int option, long long value)
{
    if (!x) return FWIME_EINVAL;
    NOT_SERVER(x);
    if (x->capturing) return FWIME_EBUSY;
    switch (option) {
    case FWIME_OPT_SHOTS_PER_BATCH: if (value < 0) break; x->opt_S = (int)value; return FWIME_OK;
    case FWIME_OPT_SEGMENT: if (value < 0) break; x->opt_K = (int)value; return FWIME_OK;
    case FWIME_OPT_PLAIN: x->opt_plain = value != 0; return FWIME_OK;
    case FWIME_OPT_GRAPH: x->opt_graph = value != 0; return FWIME_OK;
    case FWIME_OPT_HOST_IO: x->opt_host_io = value != 0; return FWIME_OK;
    case FWIME_OPT_ZCHUNK: if (value < 0 || value > 4096) break; x->opt_zchunk = (int)value; return FWIME_OK;
    case FWIME_OPT_PROFILE: x->opt_profile = value != 0; return FWIME_OK;
    case FWIME_OPT_FREE_SURFACE:
        x->opt_fs = value != 0;
        x->bg.valid = false;
        return FWIME_OK;
    case FWIME_OPT_TIME_LAG:
        if (value < 0 || value > 100000) break;
        x->opt_tlag = (int)value;
        x->bg.valid = false;
        return FWIME_OK;
    case FWIME_OPT_REUSE_BACKGROUND:
        x->opt_reuse_bg = value != 0;
        x->bg.valid = false;
        if (!x->opt_reuse_bg && x->bg.buf) {   // give the memory back
            cudaFreeAsync(x->bg.buf, x->st);
            x->bg = fwime_ctx::BgCache{};
        }
        return FWIME_OK;
    default: break;
    }
    return fail(x, FWIME_EINVAL, "bad option %d = %lld", option, value);
}

int fwime_get_option(fwime_ctx *x, int option, long long *value)
{
    if (!x || !value) return FWIME_EINVAL;
    NOT_SERVER(x);
    switch (option) {
    case FWIME_OPT_SHOTS_PER_BATCH: *value = x->opt_S; return FWIME_OK;
    case FWIME_OPT_SEGMENT: *value = x->opt_K; return FWIME_OK;
    case FWIME_OPT_PLAIN: *value = x->opt_plain; return FWIME_OK;
    case FWIME_OPT_GRAPH: *value = x->opt_graph; return FWIME_OK;
    case FWIME_OPT_HOST_IO: *value = x->opt_host_io; return FWIME_OK;
    case FWIME_OPT_ZCHUNK: *value = x->opt_zchunk; return FWIME_OK;
    case FWIME_OPT_LAUNCHES: *value = x->launches; return FWIME_OK;
    case FWIME_OPT_WORKSPACE: *value = (long long)x->ws_bytes; return FWIME_OK;
    case FWIME_OPT_PROFILE: *value = x->opt_profile; return FWIME_OK;
    case FWIME_OPT_REUSE_BACKGROUND: *value = x->opt_reuse_bg; return FWIME_OK;
    case FWIME_OPT_BACKGROUND_REUSED: *value = x->bg_used; return FWIME_OK;
    case FWIME_OPT_TIME_LAG: *value = x->opt_tlag; return FWIME_OK;
    case FWIME_OPT_FREE_SURFACE: *value = x->opt_fs; return FWIME_OK;
    case FWIME_OPT_BATCH_USED: *value = x->last_S; return FWIME_OK;
    }
    return fail(x, FWIME_EINVAL, "bad option %d", option);
}

int fwime_forward(fwime_ctx *x, const float *v, const float *w, float *d)
{
    Call c{FWIME_OP_FORWARD, v, w, nullptr, nullptr, d, 0, 0.f};
    if (!x) return FWIME_EINVAL;
    return call_op(x, c, K_NONE, K_NONE, K_DATA);
}

int fwime_born(fwime_ctx *x, const float *v, const float *w, const float *dv, float *d)
{
    if (!x) return FWIME_EINVAL;
    if (!dv) return fail(x, FWIME_EINVAL, "null dv");
    Call c{FWIME_OP_BORN, v, w, dv, nullptr, d, 0, 0.f};
    return call_op(x, c, K_MODEL, K_NONE, K_DATA);
}

int fwime_born_adj(fwime_ctx *x, const float *v, const float *w, const float *d, float *dv, int accumulate)
{
    if (!x) return FWIME_EINVAL;
    if (!d) return fail(x, FWIME_EINVAL, "null data");
    Call c{FWIME_OP_BORN_ADJ, v, w, d, nullptr, dv, accumulate ? 1 : 0, 0.f};
    return call_op(x, c, K_DATA, K_NONE, K_MODEL);
}

int fwime_born_ext(fwime_ctx *x, const float *v, const float *w, const float *pt, float *d)
{
    if (!x) return FWIME_EINVAL;
    if (!pt) return fail(x, FWIME_EINVAL, "null p~");
    Call c{FWIME_OP_BORN_EXT, v, w, pt, nullptr, d, 0, 0.f};
    return call_op(x, c, K_EXT, K_NONE, K_DATA);
}

int fwime_born_ext_adj(fwime_ctx *x, const float *v, const float *w, const float *d, float *pt, int accumulate)
{
    if (!x) return FWIME_EINVAL;
    if (!d) return fail(x, FWIME_EINVAL, "null data");
    Call c{FWIME_OP_BORN_EXT_ADJ, v, w, d, nullptr, pt, accumulate ? 1 : 0, 0.f};
    return call_op(x, c, K_DATA, K_NONE, K_EXT);
}

int fwime_tomo(fwime_ctx *x, const float *v, const float *w, const float *pt, const float *dv, float *d)
{
    if (!x) return FWIME_EINVAL;
    if (!pt || !dv) return fail(x, FWIME_EINVAL, "null p~ or dv");
    Call c{FWIME_OP_TOMO, v, w, pt, dv, d, 0, 0.f};
    return call_op(x, c, K_EXT, K_MODEL, K_DATA);
}

int fwime_tomo_adj(fwime_ctx *x, const float *v, const float *w, const float *pt, const float *d, float *dv,
                   int accumulate)
{
    if (!x) return FWIME_EINVAL;
    if (!pt || !d) return fail(x, FWIME_EINVAL, "null p~ or data");
    Call c{FWIME_OP_TOMO_ADJ, v, w, pt, d, dv, accumulate ? 1 : 0, 0.f};
    return call_op(x, c, K_EXT, K_DATA, K_MODEL);
}

int fwime_gradient(fwime_ctx *x, const float *v, const float *w, const float *pt, const float *dobs, float eps,
                   float *grad, double *objective)
{
    if (!x) return FWIME_EINVAL;
    if (!pt || !dobs) return fail(x, FWIME_EINVAL, "null p~ or observed data");
    if (!(eps >= 0.f)) return fail(x, FWIME_EINVAL, "eps must be >= 0");
    x->user_J = objective;
    Call c{FWIME_OP_GRADIENT, v, w, pt, dobs, grad, 0, eps};
    return call_op(x, c, K_EXT, K_DATA, K_MODEL);
}

int fwime_gradient_forward(fwime_ctx *x, const float *v, const float *w, const float *pt, const float *dobs, float eps,
                           double *objective)
{
    if (!x) return FWIME_EINVAL;
    NOT_SERVER(x);
    if (!v || !w || !pt || !dobs || !objective) return fail(x, FWIME_EINVAL, "null argument");
    if (!(eps >= 0.f)) return fail(x, FWIME_EINVAL, "eps must be >= 0");
    if (x->opt_host_io || x->capturing) return fail(x, FWIME_EINVAL, "the split gradient takes device pointers, no capture");
    x->launches = 0;
    x->user_J = objective;
    x->gs.valid = false;
    const int K = seg_K(x);
    if (x->opt_tlag > 0 || x->opt_plain || !gs_reserve(x, K)) {
        // no room for the state (or a schedule that places its checkpoints otherwise): the objective alone;
        // the adjoint half then runs the whole gradient
        gs_release(x);
        const int rc = enqueue_noted(x, Call{FWIME_OP_OBJECTIVE, v, w, pt, dobs, nullptr, 0, eps});
        if (rc != FWIME_OK) x->user_J = nullptr;
        return rc;
    }
    const int rc = enqueue_noted(x, Call{OP_GRAD_FWD, v, w, pt, dobs, nullptr, 0, eps});
    if (rc != FWIME_OK) {
        x->user_J = nullptr;
        gs_release(x);
        return rc;
    }
    x->gs.valid = true;
    x->gs.v = v; x->gs.w = w; x->gs.pt = pt; x->gs.K = K;
    return FWIME_OK;
}

int fwime_gradient_backward(fwime_ctx *x, const float *v, const float *w, const float *pt, const float *dobs, float eps,
                            float *grad, int accumulate)
{
    if (!x) return FWIME_EINVAL;
    NOT_SERVER(x);
    if (!v || !w || !pt || !dobs || !grad) return fail(x, FWIME_EINVAL, "null argument");
    if (!(eps >= 0.f)) return fail(x, FWIME_EINVAL, "eps must be >= 0");
    if (x->opt_host_io || x->capturing) return fail(x, FWIME_EINVAL, "the split gradient takes device pointers, no capture");
    x->launches = 0;
    const bool from_state = x->gs.valid && x->gs.buf && x->gs.v == v && x->gs.w == w && x->gs.pt == pt &&
                            x->gs.K == seg_K(x) && x->opt_tlag == 0 && !x->opt_plain;
    int rc;
    if (from_state) {
        rc = enqueue_noted(x, Call{OP_GRAD_BWD, v, w, pt, dobs, grad, accumulate ? 1 : 0, eps});
    } else {
        // the whole gradient (forward sweep recomputed); its objective is not reported
        rc = enqueue_noted(x, Call{FWIME_OP_GRADIENT, v, w, pt, dobs, grad, accumulate ? 1 : 0, eps});
    }
    x->bg_used = from_state;
    gs_release(x);   // stream-ordered: freed after the adjoint sweep that reads it
    return rc;
}

int fwime_vp_solve(fwime_ctx *x, const float *v, const float *w, const float *dres, float eps, int niter, float *pt,
                   double *history)
{
    if (!x) return FWIME_EINVAL;
    NOT_SERVER(x);
    if (!v || !w || !dres || !pt || niter < 0 || !(eps >= 0.f)) return fail(x, FWIME_EINVAL, "vp_solve arguments");
    if (x->opt_host_io || x->capturing) return fail(x, FWIME_EINVAL, "vp_solve takes device pointers, no capture");
    x->launches = 0;
    const size_t nm = (size_t)x->g.nh * x->g.nz * x->g.nx, nd = (size_t)x->nshot * x->g.nt * x->nrec;
    const long long PP = (long long)x->g.nz * x->g.nx;
    float *r = nullptr, *pdir = nullptr, *hp = nullptr, *dtmp = nullptr;
    double *sc = nullptr, *hist = nullptr;
    const int nred = 1024;
    const float eps2 = eps * eps;
    auto dot = [&](const float *a, const float *b, size_t n, double *out, double scale, int acc) -> int {
        LAUNCH(FWIME_K_OTHER, 8.0 * n, launch_dot(a, b, (long long)n, x->d_part, nred, out, acc, scale, x->st));
        return FWIME_OK;
    };
    // H q = B~* B~ q + eps^2 D^2 q  (Eq. 3)
    auto apply_H = [&](const float *q, float *out) -> int {
        TRY(enqueue_noted(x, Call{FWIME_OP_BORN_EXT, v, w, q, nullptr, dtmp, 0, 0.f}));
        TRY(enqueue_noted(x, Call{FWIME_OP_BORN_EXT_ADJ, v, w, dtmp, nullptr, out, 0, 0.f}));
        LAUNCH(FWIME_K_OTHER, 12.0 * nm, launch_dso_add(q, out, x->g.nh, PP, eps2, x->st));
        return FWIME_OK;
    };
    auto solve = [&]() -> int {
        CK(cudaMallocAsync(reinterpret_cast<void **>(&r), nm * sizeof(float), x->st));
        CK(cudaMallocAsync(reinterpret_cast<void **>(&pdir), nm * sizeof(float), x->st));
        CK(cudaMallocAsync(reinterpret_cast<void **>(&hp), nm * sizeof(float), x->st));
        CK(cudaMallocAsync(reinterpret_cast<void **>(&dtmp), nd * sizeof(float), x->st));
        CK(cudaMallocAsync(reinterpret_cast<void **>(&sc), 8 * sizeof(double), x->st));
        CK(cudaMallocAsync(reinterpret_cast<void **>(&hist), (niter + 1) * sizeof(double), x->st));
        const double consts[8] = {0, 0, 0, 0, 0, 0, 1.0, -1.0};   // sc[6] = 1, sc[7] = -1
        CK(cudaMemcpyAsync(sc, consts, sizeof(consts), cudaMemcpyHostToDevice, x->st));
        // r0 = B~* (dres - B~ p0) - eps^2 D^2 p0,  Phi(p0) = 1/2 ||B~ p0 - dres||^2 + eps^2/2 ||D p0||^2
        TRY(enqueue_noted(x, Call{FWIME_OP_BORN_EXT, v, w, pt, nullptr, dtmp, 0, 0.f}));
        LAUNCH(FWIME_K_OTHER, 12.0 * nd, launch_axpby_dev(dtmp, dres, (long long)nd, sc, 6, 1.f, 7, x->st));   // dres - B~ p0
        TRY(dot(dtmp, dtmp, nd, sc + 5, 0.5, 0));
        LAUNCH(FWIME_K_OTHER, 4.0 * nm, launch_dso(pt, x->g.nh, PP, x->d_part, nred, x->st));
        LAUNCH(FWIME_K_OTHER, 8.0, launch_sum_partials(x->d_part, nred, sc + 5, 1, 0.5 * (double)eps2, x->st));
        TRY(enqueue_noted(x, Call{FWIME_OP_BORN_EXT_ADJ, v, w, dtmp, nullptr, r, 0, 0.f}));
        LAUNCH(FWIME_K_OTHER, 12.0 * nm, launch_dso_add(pt, r, x->g.nh, PP, -eps2, x->st));
        CK(cudaMemcpyAsync(pdir, r, nm * sizeof(float), cudaMemcpyDeviceToDevice, x->st));
        TRY(dot(r, r, nm, sc + 0, 1.0, 0));
        CK(cudaMemcpyAsync(hist, sc + 5, sizeof(double), cudaMemcpyDeviceToDevice, x->st));
        for (int k = 0; k < niter; ++k) {
            TRY(apply_H(pdir, hp));
            TRY(dot(pdir, hp, nm, sc + 1, 1.0, 0));                              // p.Hp
            LAUNCH(FWIME_K_OTHER, 8.0, launch_cg_scalars(sc, 0, hist, k + 1, x->st));   // alpha; Phi -= alpha rr / 2
            LAUNCH(FWIME_K_OTHER, 12.0 * nm, launch_axpby_dev(pt, pdir, (long long)nm, sc, 2, 1.f, -1, x->st));   // p~ += alpha p
            LAUNCH(FWIME_K_OTHER, 12.0 * nm, launch_axpby_dev(r, hp, (long long)nm, sc, 2, -1.f, -1, x->st));     // r -= alpha Hp
            TRY(dot(r, r, nm, sc + 4, 1.0, 0));
            LAUNCH(FWIME_K_OTHER, 8.0, launch_cg_scalars(sc, 1, nullptr, 0, x->st));     // beta = rr_new / rr
            LAUNCH(FWIME_K_OTHER, 12.0 * nm, launch_axpby_dev(pdir, r, (long long)nm, sc, 6, 1.f, 3, x->st));   // p = r + beta p
        }
        return FWIME_OK;
    };
    // v and w cannot change during the solve: every B~* starts from the checkpoints of the B~ before it
    const int saved_reuse = x->opt_reuse_bg;
    x->opt_reuse_bg = 1;
    const int rc = solve();
    x->opt_reuse_bg = saved_reuse;
    x->bg.valid = false;
    if (!saved_reuse && x->bg.buf) {
        cudaFreeAsync(x->bg.buf, x->st);
        x->bg = fwime_ctx::BgCache{};
    }
    for (void *q : {(void *)r, (void *)pdir, (void *)hp, (void *)dtmp, (void *)sc})
        if (q) cudaFreeAsync(q, x->st);
    if (rc != FWIME_OK) {
        if (hist) cudaFreeAsync(hist, x->st);
        return rc;
    }
    if (x->vp_hist_dev) CK(cudaFreeAsync(x->vp_hist_dev, x->st));   // an earlier solve's history, never synced
    x->vp_hist_dev = hist;
    x->vp_hist_user = history;
    x->vp_hist_n = niter + 1;
    return FWIME_OK;
}

int fwime_spline(fwime_ctx *x, int nzs, const float *zs, int nxs, const float *xs, const float *in, float *out,
                 int adjoint, int accumulate)
{
    if (!x) return FWIME_EINVAL;
    NOT_SERVER(x);
    if (nzs < 1 || nxs < 1 || !zs || !xs || !in || !out) return fail(x, FWIME_EINVAL, "spline arguments");
    if (x->opt_host_io || x->capturing) return fail(x, FWIME_EINVAL, "spline takes device pointers, no capture");
    for (int i = 0; i < nzs; ++i)
        if (!std::isfinite(zs[i]) || (i && !(zs[i] > zs[i - 1]))) return fail(x, FWIME_EINVAL, "zs must increase");
    for (int i = 0; i < nxs; ++i)
        if (!std::isfinite(xs[i]) || (i && !(xs[i] > xs[i - 1]))) return fail(x, FWIME_EINVAL, "xs must increase");
    x->launches = 0;
    float *dn = nullptr;
    const size_t nn = (size_t)nzs + nxs, nt = adjoint ? (size_t)x->g.nz * nxs : 0;
    CK(cudaMallocAsync(reinterpret_cast<void **>(&dn), (nn + nt) * sizeof(float), x->st));
    int rc = FWIME_OK;
    cudaError_t e = cudaMemcpyAsync(dn, zs, nzs * sizeof(float), cudaMemcpyHostToDevice, x->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dn + nzs, xs, nxs * sizeof(float), cudaMemcpyHostToDevice, x->st);
    if (e != cudaSuccess) rc = fail(x, FWIME_ECUDA, "spline nodes: %s", cudaGetErrorString(e));
    if (rc == FWIME_OK) {
        auto go = [&]() -> int {
            LAUNCH(FWIME_K_OTHER, 4.0 * ((double)x->g.nz * x->g.nx + (double)nzs * nxs) * (adjoint ? 2 : 1),
                   launch_spline(dn, nzs, dn + nzs, nxs, x->g.nz, x->g.nx, x->g.dz, x->g.dx, in, out,
                                 dn + nn, adjoint, accumulate, x->st));
            return FWIME_OK;
        };
        rc = go();
    }
    cudaFreeAsync(dn, x->st);
    return rc;
}

int fwime_spline_refine(fwime_ctx *x, int nzc, const float *zc, int nxc, const float *xc, const float *mc, int nzf,
                        const float *zf, int nxf, const float *xf, float *mf)
{
    if (!x) return FWIME_EINVAL;
    NOT_SERVER(x);
    if (nzc < 1 || nxc < 1 || nzf < 1 || nxf < 1 || !zc || !xc || !zf || !xf || !mc || !mf)
        return fail(x, FWIME_EINVAL, "spline_refine arguments");
    if (x->opt_host_io || x->capturing) return fail(x, FWIME_EINVAL, "spline_refine takes device pointers, no capture");
    const int n[4] = {nzc, nxc, nzf, nxf};
    const float *nodes[4] = {zc, xc, zf, xf};
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < n[a]; ++i)
            if (!std::isfinite(nodes[a][i]) || (i && !(nodes[a][i] > nodes[a][i - 1])))
                return fail(x, FWIME_EINVAL, "spline nodes must be finite and increase");
    x->launches = 0;
    float *dn = nullptr;
    const size_t nn = (size_t)nzc + nxc + nzf + nxf;
    CK(cudaMallocAsync(reinterpret_cast<void **>(&dn), nn * sizeof(float), x->st));
    int rc = FWIME_OK;
    size_t off = 0;
    for (int a = 0; a < 4 && rc == FWIME_OK; ++a) {
        const cudaError_t e = cudaMemcpyAsync(dn + off, nodes[a], n[a] * sizeof(float), cudaMemcpyHostToDevice, x->st);
        if (e != cudaSuccess) rc = fail(x, FWIME_ECUDA, "spline nodes: %s", cudaGetErrorString(e));
        off += n[a];
    }
    if (rc == FWIME_OK) {
        auto go = [&]() -> int {
            LAUNCH(FWIME_K_OTHER, 4.0 * ((double)nzc * nxc + (double)nzf * nxf),
                   launch_spline_refine(dn, nzc, dn + nzc, nxc, mc, dn + nzc + nxc, nzf, dn + nzc + nxc + nzf, nxf, mf,
                                        x->st));
            return FWIME_OK;
        };
        rc = go();
    }
    cudaFreeAsync(dn, x->st);   // (copies from pageable host memory return once the source has been staged)
    return rc;
}

int fwime_forward_group(fwime_ctx *const *ctxs, int n, const float *const *v, const float *const *w, float *const *d)
{
    if (!ctxs || !v || !w || !d || n < 1 || n > 4096) return FWIME_EINVAL;
    fwime_ctx *x = ctxs[0];
    if (!x) return FWIME_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !v[i] || !w[i] || !d[i]) return fail(x, FWIME_EINVAL, "null member %d", i);
        if (ctxs[i]->srv) return fail(x, FWIME_EINVAL, "member %d is a server context", i);
        if (ctxs[i]->st != x->st) return fail(x, FWIME_EINVAL, "group members must share one stream");
        if (ctxs[i]->capturing || ctxs[i]->opt_host_io) return fail(x, FWIME_EINVAL, "member %d: capture/host I/O", i);
        if (ctxs[i]->opt_fs) return fail(x, FWIME_EINVAL, "member %d: the grouped forward has no free surface", i);
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(x, FWIME_EINVAL, "member %d repeats member %d", i, j);
    }
    x->launches = 0;
    std::vector<Run> runs(n);
    for (int i = 0; i < n; ++i) {
        fwime_ctx *m = ctxs[i];
        TRY(plan(m, FWIME_OP_FORWARD, runs[i].w));
        if (runs[i].w.S < m->nshot)
            return fail(x, FWIME_ENOMEM, "group member %d: %d shots do not fit one batch", i, m->nshot);
        init_run(m, runs[i], m->nshot);
        const long long before = m->launches;
        TRY(prep_model(m, runs[i], v[i]));
        if (m != x) x->launches += m->launches - before;   // the group's count includes every member's prep
        TRY(zero(m, runs[i].w.f[0], sizeof(float) * m->nshot * m->P));
        TRY(zero(m, runs[i].w.f[1], sizeof(float) * m->nshot * m->P));
        TRY(zero(m, d[i], sizeof(float) * (size_t)m->nshot * m->g.nt * m->nrec));
    }
    // members in decreasing nt: the ones still running at a step are a prefix
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ctxs[a]->g.nt > ctxs[b]->g.nt; });
    std::vector<GroupMember> gm(n);
    std::vector<GroupRec> gr(n);
    std::vector<int> cta_end(n), rec_end(n);
    int ctas = 0, recs = 0;
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        fwime_ctx *m = ctxs[i];
        Run &r = runs[i];
        PropArgs a = r.base;
        a.c = r.w.c; a.gz = r.w.gz; a.gx = r.w.gx; a.d2 = nullptr;
        a.src_off = m->d_src_off; a.src_amp = w[i]; a.src_stride = m->g.nt;
        a.f0 = a.f1 = a.f2 = a.coef = a.fc = nullptr;
        a.naux_max = 2;
        prop_pairs(a);
        gm[k].a[0] = a; gm[k].a[0].cur = r.w.f[0]; gm[k].a[0].prev = r.w.f[1]; gm[k].a[0].out = r.w.f[1];
        gm[k].a[1] = a; gm[k].a[1].cur = r.w.f[1]; gm[k].a[1].prev = r.w.f[0]; gm[k].a[1].out = r.w.f[0];
        gm[k].ctas_per_shot = (r.nstrip * r.nchunk + PROP_WARPS - 1) / PROP_WARPS;
        gm[k].cta_begin = ctas;
        ctas += gm[k].ctas_per_shot * m->nshot;
        cta_end[k] = ctas;
        gr[k].rec_off = m->d_rec_off; gr[k].fA = r.w.f[0]; gr[k].fB = r.w.f[1]; gr[k].d = d[i]; gr[k].P = m->P;
        gr[k].nrec = m->nrec; gr[k].nshot = m->nshot; gr[k].nt = m->g.nt; gr[k].rec_begin = recs;
        recs += m->nshot * m->nrec;
        rec_end[k] = recs;
    }
    void *dev = nullptr;
    const size_t bytes = n * (sizeof(GroupMember) + sizeof(GroupRec));
    CK(cudaMallocAsync(&dev, bytes, x->st));
    std::vector<char> host(bytes);
    std::memcpy(host.data(), gm.data(), n * sizeof(GroupMember));
    std::memcpy(host.data() + n * sizeof(GroupMember), gr.data(), n * sizeof(GroupRec));
    CK(cudaMemcpyAsync(dev, host.data(), bytes, cudaMemcpyHostToDevice, x->st));
    CK(cudaStreamSynchronize(x->st));   // the host copy of the tables is a local
    const GroupMember *dgm = reinterpret_cast<const GroupMember *>(dev);
    const GroupRec *dgr = reinterpret_cast<const GroupRec *>(reinterpret_cast<char *>(dev) + n * sizeof(GroupMember));
    const int maxnt = ctxs[order[0]]->g.nt;
    int nactive = n;
    for (int step = 0; step + 1 < maxnt; ++step) {
        while (nactive > 0 && ctxs[order[nactive - 1]]->g.nt - 1 <= step) --nactive;
        double pts = 0.0;
        for (int k = 0; k < nactive; ++k) pts += (double)ctxs[order[k]]->nshot * ctxs[order[k]]->NZ * ctxs[order[k]]->NX;
        LAUNCH(FWIME_K_PROP, 12.0 * pts, launch_prop_group(dgm, nactive, cta_end[nactive - 1], dgr, 0, step, x->st, false));
        LAUNCH(FWIME_K_POINTS, 8.0 * rec_end[nactive - 1],
               launch_prop_group(dgm, nactive, 0, dgr, rec_end[nactive - 1], step, x->st, true));
    }
    CK(cudaFreeAsync(dev, x->st));
    return FWIME_OK;
}

// Stencil chunking (rows per warp) for launches of S shots: every candidate of a ladder and the chunkings
// that come closest to whole waves of resident warps, timed on the plain variant (reps launches after one
// warm-up, two passes, the faster kept).  Times within 1 % are noise at this length, so among them the
// chunking whose last wave is fullest wins (a partly filled last wave idles SMs in every launch, which a
// long run of launches shows more than the timing does).
static int pick_zchunk(fwime_ctx *x, Run &r, int S, std::vector<int> cand, int reps, float *us_out)
{
    const int rows = x->NZ - 8;
    const long long per_chunk = (long long)((x->NXP + STRIP - 1) / STRIP) * S;   // warps per chunk row
    long long resident = 0;
    int bps = 0, nsm = 0, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && prop_occupancy(&bps) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && bps > 0) {
        resident = (long long)bps * nsm * PROP_WARPS;
        for (int waves = 1; waves <= 12; ++waves) {
            const long long nchunk = (waves * resident) / per_chunk;
            if (nchunk < 1) continue;
            const int zc = (int)((rows + nchunk - 1) / nchunk);
            if (zc >= 4 && zc <= 512) cand.push_back(zc);
        }
    }
    cudaGetLastError();
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    while (cand.size() > 1 && cand.back() > rows) cand.pop_back();
    auto fill = [&](int zc) {   // used fraction of the launch's waves of resident warps
        if (resident <= 0) return 1.0;
        const double w = (double)per_chunk * ((rows + zc - 1) / zc) / (double)resident;
        return w / std::ceil(w);
    };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 0;
    }
    std::vector<float> us(cand.size(), 1e30f);
    int rc = FWIME_OK;
    for (int pass = 0; pass < 2 && rc == FWIME_OK; ++pass) {
        for (size_t i = 0; i < cand.size() && rc == FWIME_OK; ++i) {
            x->opt_zchunk = cand[i];
            init_run(x, r, S);
            rc = prop(r, S, r.w.f[0], r.w.f[1], r.w.f[1], nullptr, nullptr, 0);
            if (rc != FWIME_OK) break;
            float ms = 0.f;
            if (cudaEventRecord(e0, x->st) != cudaSuccess) { rc = FWIME_ECUDA; break; }
            for (int it = 0; it < reps && rc == FWIME_OK; ++it)
                rc = prop(r, S, r.w.f[0], r.w.f[1], r.w.f[1], nullptr, nullptr, 0);
            if (rc != FWIME_OK) break;
            if (cudaEventRecord(e1, x->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = FWIME_ECUDA;
                break;
            }
            us[i] = std::min(us[i], 1e3f * ms / reps);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FWIME_OK) return 0;
    float best = 1e30f;
    for (float u : us) best = std::min(best, u);
    size_t pi = cand.size();
    for (size_t i = 0; i < cand.size(); ++i) {
        if (us[i] > 1.01f * best) continue;
        const double df = pi == cand.size() ? 1.0 : fill(cand[i]) - fill(cand[pi]);
        if (df > 1e-9 || (df > -1e-9 && us[i] < us[pi])) pi = i;
    }
    if (us_out) *us_out = us[pi];
    return cand[pi];
}

int fwime_autotune(fwime_ctx *x, int op, int *zchunk_out, float *us_per_launch_out)
{
    if (!x || op < 0 || op > FWIME_OP_OBJECTIVE) return FWIME_EINVAL;
    NOT_SERVER(x);
    if (x->capturing) return FWIME_EBUSY;
    Run r;
    TRY(plan(x, op, r.w));
    const int S = r.w.S;
    // timing needs no model: zero c, the sponge tables and two batch fields
    TRY(zero(x, r.w.c, sizeof(float) * x->P));
    TRY(zero(x, r.w.gz, sizeof(float) * x->NZ));
    TRY(zero(x, r.w.gx, sizeof(float) * x->NXP));
    TRY(zero(x, r.w.f[0], sizeof(float) * S * x->P));
    TRY(zero(x, r.w.f[1], sizeof(float) * S * x->P));
    const int saved = x->opt_zchunk, saved_prof = x->opt_profile;
    x->opt_profile = 0;
    float best_us = 0.f;
    const int best = pick_zchunk(x, r, S, {8, 16, 24, 32, 48, 64, 96, 128, 192, 256}, 6, &best_us);
    x->opt_profile = saved_prof;
    x->opt_zchunk = best > 0 ? best : saved;
    if (best == 0) return fail(x, FWIME_ECUDA, "stencil chunking timing failed");
    if (zchunk_out) *zchunk_out = x->opt_zchunk;
    if (us_per_launch_out) *us_per_launch_out = best_us;
    return FWIME_OK;
}

// Schedule autotuner: segment length K x shots per launch S x stencil chunking, timed on this device.
// For each K (the automatic one, half, double) the planner gives the largest equal batch S_K that fits;
// S_K and half of it are tried.  At each (K, S) the stencil is timed for its chunking candidates and the
// operator's extension kernels once over a full segment of K x S pairs; the modelled time per shot,
//   (nt - 1) * props * t_stencil / S + nseg * (scatters * t_scatter + images * t_image) / S,
// picks the schedule (props, scatters, images: the operator's launches per step and per segment).
int fwime_autotune_schedule(fwime_ctx *x, int op, fwime_schedule *res)
{
    if (!x || !res || op < 0 || op > FWIME_OP_OBJECTIVE) return FWIME_EINVAL;
    NOT_SERVER(x);
    if (x->capturing) return FWIME_EBUSY;
    if (x->opt_plain) return fail(x, FWIME_EINVAL, "the plain path has a fixed schedule");
    static const int PROPS[] = {1, 2, 3, 2, 3, 4, 6, 6, 2};
    static const int SCAT[] = {0, 0, 0, 1, 0, 3, 2, 2, 1};
    static const int IMGS[] = {0, 0, 0, 0, 1, 0, 1, 1, 0};
    const bool lag = x->opt_tlag > 0;   // the time-lag schedules: extension kernels not timed here
    const int saved_K = x->opt_K, saved_S = x->opt_S, saved_zc = x->opt_zchunk, saved_prof = x->opt_profile;
    x->opt_profile = 0;
    std::vector<int> Ks;
    if (saved_K > 0) Ks = {saved_K};
    else {
        const int K0 = seg_K(x);
        Ks = {K0, std::max(K0 / 2, 8), std::min(2 * K0, x->g.nt - 1)};
        std::sort(Ks.begin(), Ks.end());
        Ks.erase(std::unique(Ks.begin(), Ks.end()), Ks.end());
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        x->opt_profile = saved_prof;
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(x, FWIME_ECUDA, "autotune events");
    }
    auto timed = [&](auto &&body, int reps, float &us) -> int {
        for (int it = 0; it < 1; ++it) TRY(body());
        CK(cudaEventRecord(e0, x->st));
        for (int it = 0; it < reps; ++it) TRY(body());
        CK(cudaEventRecord(e1, x->st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        us = 1e3f * ms / reps;
        return FWIME_OK;
    };
    double best = 1e300;
    fwime_schedule out{};
    int rc = FWIME_OK;
    for (int K : Ks) {
        x->opt_K = K;
        x->opt_S = 0;
        Run r;
        rc = plan(x, op, r.w);
        if (rc != FWIME_OK) { rc = FWIME_OK; continue; }   // this K does not fit: skip it
        const int SK = r.w.S;
        std::vector<int> Ss = {SK};
        if (SK > 1) {
            const int nb = (x->nshot + SK - 1) / SK;
            Ss.push_back((x->nshot + 2 * nb - 1) / (2 * nb));
        }
        for (int S : Ss) {
            x->opt_S = S;
            rc = plan(x, op, r.w);
            if (rc != FWIME_OK) break;
            const long long SP = (long long)S * x->P;
            // timing needs no model: zeros everywhere the kernels read
            rc = zero(x, x->ws, x->ws_bytes);
            if (rc != FWIME_OK) break;
            // stencil: the chunking candidates (a ladder and whole waves of resident warps)
            float tp = 0.f;
            const int zbest = pick_zchunk(x, r, S, {16, 32, 48, 64, 96, 128}, 4, &tp);
            if (zbest == 0) { rc = fail(x, FWIME_ECUDA, "stencil chunking timing failed"); break; }
            x->opt_zchunk = zbest;
            init_run(x, r, S);
            const int kk = std::min(K, x->g.nt - 1);
            float tsc = 0.f, tim = 0.f;
            if (!lag && SCAT[op] > 0 && r.w.W && r.w.ring[0] && r.w.ring[1]) {
                rc = timed([&]() {
                    return scatter(r, S, 0, kk, r.w.W, ringref(r.w.ring[0], SP, 0, 0), ringref(r.w.ring[1], SP, 0, 0),
                                   +1, 0);
                }, 2, tsc);
                if (rc != FWIME_OK) break;
            }
            float *img_acc = op == FWIME_OP_BORN_EXT_ADJ ? r.w.acc1 : r.w.acc2;
            float *lring = op == FWIME_OP_BORN_EXT_ADJ ? r.w.ring[1] : r.w.ring[3];
            if (!lag && IMGS[op] > 0 && img_acc && r.w.ring[0] && lring) {
                rc = timed([&]() {
                    return image(r, S, 0, kk, IMG_EXT, ringref(r.w.ring[0], SP, 0, 0), ringref(lring, SP, r.w.R, 1),
                                 ringref(nullptr, 0, 0, 0), ringref(nullptr, 0, 0, 0), 1.f, nullptr, img_acc);
                }, 2, tim);
                if (rc != FWIME_OK) break;
            }
            const double nseg = (double)r.w.nseg;
            const double per_shot = ((double)(x->g.nt - 1) * PROPS[op] * tp + nseg * (SCAT[op] * tsc + IMGS[op] * tim)) / S;
            if (per_shot < best) {
                best = per_shot;
                out.shots_per_batch = S;
                out.segment = K;
                out.zchunk = zbest;
                out.us_stencil = tp;
                out.us_scatter = tsc;
                out.us_image = tim;
                out.us_per_shot = per_shot;
            }
        }
        if (rc != FWIME_OK) break;
    }
    cleanup();
    if (rc != FWIME_OK || best >= 1e299) {
        x->opt_K = saved_K; x->opt_S = saved_S; x->opt_zchunk = saved_zc;
        return rc != FWIME_OK ? rc : fail(x, FWIME_ENOMEM, "no schedule fits");
    }
    x->opt_K = out.segment;
    x->opt_S = out.shots_per_batch;
    x->opt_zchunk = out.zchunk;
    *res = out;
    return FWIME_OK;
}

int fwime_objective(fwime_ctx *x, const float *v, const float *w, const float *pt, const float *dobs, float eps,
                    double *objective)
{
    if (!x) return FWIME_EINVAL;
    if (!pt || !dobs || !objective) return fail(x, FWIME_EINVAL, "null p~, observed data or objective");
    if (!(eps >= 0.f)) return fail(x, FWIME_EINVAL, "eps must be >= 0");
    x->user_J = objective;
    Call c{FWIME_OP_OBJECTIVE, v, w, pt, dobs, nullptr, 0, eps};
    return call_op(x, c, K_EXT, K_DATA, K_NONE);
}

int fwime_sync(fwime_ctx *x)
{
    if (!x) return FWIME_EINVAL;
    if (x->srv) return server_sync(x->srv);
    CK(x->st ? cudaStreamSynchronize(x->st) : cudaDeviceSynchronize());
    TRY(prof_collect(x));
    CK(cudaMemcpyAsync(x->h_status, x->d_status, sizeof(int), cudaMemcpyDeviceToHost, x->st));
    CK(cudaStreamSynchronize(x->st));
    const int st = *x->h_status;
    if (st) CK(cudaMemsetAsync(x->d_status, 0, sizeof(int), x->st));
    if (x->user_J) {
        *x->user_J = *x->h_J;
        x->user_J = nullptr;
    }
    if (x->vp_hist_dev) {
        if (x->vp_hist_user)
            CK(cudaMemcpy(x->vp_hist_user, x->vp_hist_dev, x->vp_hist_n * sizeof(double), cudaMemcpyDeviceToHost));
        CK(cudaFreeAsync(x->vp_hist_dev, x->st));
        x->vp_hist_dev = x->vp_hist_user = nullptr;
    }
    if (st & ST_CFL) return fail(x, FWIME_ECFL, "velocity violates the CFL bound or is not positive");
    return FWIME_OK;
}

int fwime_profile_read(fwime_ctx *x, int kernel, double *ms, long long *launches, double *bytes, int reset)
{
    if (!x || kernel < 0 || kernel > FWIME_K_OTHER) return FWIME_EINVAL;
    NOT_SERVER(x);
    TRY(prof_collect(x));
    if (ms) *ms = x->prof_ms[kernel];
    if (launches) *launches = x->prof_n[kernel];
    if (bytes) *bytes = x->prof_bytes[kernel];
    if (reset)
        for (int k = 0; k < 5; ++k) { x->prof_ms[k] = 0; x->prof_bytes[k] = 0; x->prof_n[k] = 0; }
    return FWIME_OK;
}

int fwime_last_error_detail(fwime_ctx *x, char *buf, size_t n)
{
    if (!x || !buf || n == 0) return FWIME_EINVAL;
    snprintf(buf, n, "%s", x->err);
    return FWIME_OK;
}

}  // extern "C"
