// api.cu -- host side of the C ABI declared in include/qsg.h: validation,
// workspace carving, acceptance tables, and the ordering of kernel launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qsg.h"
#include "qsg_launch.h"

using namespace qsg;

static std::atomic<unsigned long long> g_launches{0};
void qsg::count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

namespace {

// NVTX range over one entry point (visible in Nsight timelines; costs nothing
// when no tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

constexpr size_t kAlign = 256;
constexpr int kMaxA = 16384;               // longest A_i table of the tempering test
constexpr size_t kScratchCap = 1024u << 20;  // bytes of correlator scratch (transposed bits, E4M3 rows)

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool valid_shape(const qsg_shape &s) {
    if (s.L < 2 || s.L > 32 || (s.L & 1)) return false;
    if (s.Ltau < 2 || s.Ltau > 65536 || (s.Ltau & 1)) return false;
    if (s.n_samples < 1 || s.n_replicas < 1 || s.n_replicas > 1023 || s.n_k < 1 || s.n_k > 128) return false;
    if (s.algo != QSG_METROPOLIS && s.algo != QSG_HEATBATH) return false;
    if (s.boundary != QSG_PBC && s.boundary != QSG_APBC) return false;
    if (s.reserved != 0) return false;
    const double words = (double)((s.n_samples + 63) / 64) * s.n_replicas * s.n_k * (double)s.L * s.L * s.Ltau;
    return words < 4.0e10;
}

Group describe(const qsg_shape &s, int gid) {
    Group g;
    std::memset(&g, 0, sizeof(g));
    g.L = s.L;
    g.Ltau = s.Ltau;
    g.W = (s.n_samples + 63) / 64;
    g.R = s.n_replicas;
    g.K = s.n_k;
    g.algo = s.algo;
    g.boundary = s.boundary;
    g.gid = gid;
    g.N = s.L * s.L * s.Ltau;
    g.nslots = g.W * g.R * g.K;
    g.nlag = s.Ltau / 2 + 1;
    g.n_samples = s.n_samples;
    g.nwx = (s.L * s.L + 63) / 64;
    g.xi_norm = 2.0 * std::sin(3.14159265358979323846 / s.L);
    return g;
}

int a_cap(const Group &g) {
    const long long need = (6LL * g.N >> 6) + 1;
    return (int)(need < kMaxA ? need : kMaxA);
}

struct PlanBuffers {
    Group *groups = nullptr;
    int *order = nullptr, *prefix = nullptr, *chunk = nullptr;
    unsigned *queue = nullptr;
    uint32_t *sweep_base = nullptr;
};

// Walk the workspace: when base is null only the size is computed.
size_t carve(std::vector<Group> &gs, char *base, int **err, uint64_t **scratch, size_t *scratch_words,
             PlanBuffers *pb = nullptr) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off = align_up(off + bytes);
        return p;
    };
    *err = (int *)take(sizeof(int) * 4);
    size_t sw = 0;
    for (auto &g : gs) {
        g.S = (uint64_t *)take(sizeof(uint64_t) * (size_t)g.nslots * g.N);
        g.Jx = (uint64_t *)take(sizeof(uint64_t) * (size_t)g.W * g.L * g.L);
        g.Jy = (uint64_t *)take(sizeof(uint64_t) * (size_t)g.W * g.L * g.L);
        g.thr = (uint32_t *)take(sizeof(uint32_t) * 16 * g.K);
        const int np = g.K > 1 ? g.K - 1 : 1;
        g.ptA = (uint64_t *)take(sizeof(uint64_t) * (size_t)np * a_cap(g));
        g.ptA_off = (int32_t *)take(sizeof(int32_t) * np);
        g.ptA_len = (int32_t *)take(sizeof(int32_t) * np);
        g.ptB = (uint64_t *)take(sizeof(uint64_t) * 64 * np);
        g.U = (int32_t *)take(sizeof(int32_t) * 64 * (size_t)g.nslots);
        g.swapmask = (uint32_t *)take(sizeof(uint32_t) * 2 * (size_t)g.W * g.R * np);
        g.acc = (unsigned long long *)take(sizeof(unsigned long long) * (size_t)g.W * 64 * np);
        const size_t nc = (size_t)g.R * g.W * 64 * g.K * g.nlag;
        g.Cacc = (long long *)take(sizeof(long long) * nc);
        g.Qacc = (long long *)take(sizeof(long long) * nc);
        g.Pacc = (long long *)take(sizeof(long long) * (size_t)g.W * 64 * g.K);
        g.outC = (double *)take(sizeof(double) * nc);
        g.outQ = (double *)take(sizeof(double) * nc);
        g.outP = (double *)take(sizeof(double) * (size_t)g.W * 64 * g.K);
        const size_t nsk = (size_t)g.W * 64 * g.K, nd = (size_t)(g.L / 2 + 1);
        g.P4acc = (unsigned long long *)take(sizeof(unsigned long long) * 2 * nsk);
        g.T3acc = (long long *)take(sizeof(long long) * nsk);
        g.Gacc = (long long *)take(sizeof(long long) * nsk * nd);
        g.F3acc = (long long *)take(sizeof(long long) * nsk * nd);
        g.PPacc = (long long *)take(sizeof(long long) * nsk * (size_t)(g.R * (g.R - 1) / 2 + 1));
        g.outO = (double *)take(sizeof(double) * nsk * 7);
        g.outK = (double *)take(sizeof(double) * (size_t)g.K * 8);
        g.wcos = (double *)take(sizeof(double) * nd);
        g.arrivals = (unsigned *)take(sizeof(unsigned) * (size_t)g.nslots * (g.Ltau / 4 > 0 ? g.Ltau / 4 : 1));
        // one (w, j) pair at least, up to the cap
        const size_t per = measure_scratch_words_per_pair(g);
        size_t want = kScratchCap / sizeof(uint64_t);
        if (want < per) want = per;
        const size_t all = per * (size_t)g.W * g.K;
        if (want > all) want = all;
        // the scratch also holds the coupling features, [W*64][64] float
        const size_t feat = (size_t)g.W * 64 * 64 / 2;
        if (want < feat) want = feat;
        if (want > sw) sw = want;
    }
    *scratch = (uint64_t *)take(sizeof(uint64_t) * sw);
    *scratch_words = sw;
    // persistent-launch plan: group table, order, unit prefix sums, chunks, queue
    const size_t ng = gs.size();
    Group *pg = (Group *)take(sizeof(Group) * ng);
    int *po = (int *)take(sizeof(int) * ng);
    int *pp = (int *)take(sizeof(int) * (ng + 1));
    int *pc = (int *)take(sizeof(int) * ng);
    unsigned *pq = (unsigned *)take(sizeof(unsigned) * 2);
    uint32_t *psb = (uint32_t *)take(sizeof(uint32_t) * 4);
    if (pb) {
        pb->sweep_base = psb;
        pb->groups = pg;
        pb->order = po;
        pb->prefix = pp;
        pb->chunk = pc;
        pb->queue = pq;
    }
    return off;
}

// ---- acceptance tables (host FP64, integer results) ----------------------
uint32_t met_threshold(double k, int Sh) {
    const double p = std::exp(-(2.0 * k * (double)Sh));
    return (uint32_t)std::floor(p * 4294967296.0);
}

uint32_t hb_threshold(double k, int h) {
    const double p = 1.0 / (1.0 + std::exp(-(2.0 * k * (double)h)));
    double t = std::floor(p * 4294967296.0);
    if (t > 4294967295.0) t = 4294967295.0;
    return (uint32_t)t;
}

}  // namespace

bool qsg::build_accept_tables(const double *k, int K, uint32_t *table) {
    for (int j = 0; j < K; ++j) {
        if (!(k[j] > 0.0) || !(k[j] < 3.0)) return false;
        if (j > 0 && !(k[j] > k[j - 1])) return false;
        uint32_t *t = table + 16 * (size_t)j;
        for (int n = 0; n < 16; ++n) t[n] = 0u;
        for (int c = 0; c < 3; ++c) t[c] = met_threshold(k[j], 2 * (c + 1));
        for (int n = 0; n < 7; ++n) t[8 + n] = hb_threshold(k[j], 6 - 2 * n);
        for (int c = 0; c < 2; ++c)
            if (t[c] < t[c + 1]) return false;
        for (int n = 0; n < 6; ++n)
            if (t[8 + n] < t[9 + n]) return false;
    }
    return true;
}

namespace {

uint64_t pt_factor(double delta, long long n) {
    return (uint64_t)std::floor(std::exp(-(delta * (double)n)) * 4294967296.0);
}

}  // namespace

struct qsg_ctx {
    std::vector<qsg_shape> shapes;
    std::vector<Group> groups;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    int *d_err = nullptr;
    uint64_t *scratch = nullptr;
    size_t scratch_words = 0;
    cudaStream_t stream = nullptr;
    uint64_t seed = 0;
    bool initialised = false;
    bool energy_fresh = false;
    uint32_t sweeps = 0, swaps = 0;
    long long n_meas = 0;
    int sweep_kernel = 0;  // QSG_OPT_SWEEP_KERNEL
    int chunk = 0;         // QSG_OPT_CHUNK
    int corr_tensor = 1;   // QSG_OPT_CORR_KERNEL: 1 tensor cores, 0 integer pipes
    int persistent = 0;    // QSG_OPT_PERSISTENT: 0 automatic, 1 off, 2 persistent kernel, 3 one stream per group
    int triples = 1;       // QSG_OPT_ONETIME: 1 with the three-replica sums, 0 without
    int tail = 0;          // QSG_OPT_TAIL: slots swept in quarter-length chunks, last
    int upb = 0;           // QSG_OPT_UNITS_PER_BLOCK: 0 automatic, else 1, 2, 4, 8 or 16
    unsigned wait_limit = kDefaultWaitLimit;  // QSG_OPT_WAIT_LIMIT: polls per bounded device wait
    PlanBuffers pb;
    PersistentPlan plan{};
    bool plan_ok = false;
    // CUDA graph of graph_batch sweeps (QSG_OPT_GRAPH), captured on a private
    // stream and replayed on `stream`; the kernels read the sweep index from
    // pb.sweep_base, which base_valid says equals `sweeps`.
    int graph_batch = 0;
    long long graph_key = -1;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    unsigned long long graph_launches = 0;  // kernels per replay
    bool base_valid = false;
    std::string last_cuda;
    // one stream per group for the concurrent multi-group mode, with the fork
    // and join events that order them against the context's stream
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    // qsg_read_correlators_async: the point on `stream` the finish and copies
    // on the caller's stream wait for, and their completion, which every later
    // writer of the correlator buffers waits for
    cudaEvent_t fin_ev = nullptr, copy_ev = nullptr;
    bool copy_pending = false;
    int *h_flag = nullptr;  // page-locked copy of the device flag, taken with the copies
    bool flag_pending = false;
    ~qsg_ctx() {
        // the copies read the workspace, which the caller frees after this
        if (copy_pending) cudaEventSynchronize(copy_ev);
        if (fin_ev) cudaEventDestroy(fin_ev);
        if (copy_ev) cudaEventDestroy(copy_ev);
        if (h_flag) cudaFreeHost(h_flag);
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (cudaStream_t t : side) cudaStreamDestroy(t);
        for (cudaEvent_t e : joins) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
    }
};

static qsg_status cuda_fail(qsg_ctx *c, cudaError_t e) {
    if (e == cudaSuccess) return QSG_OK;
    c->last_cuda = cudaGetErrorString(e);
    return QSG_ERR_CUDA;
}

#define QSG_CUDA(c, expr)                                  \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return cuda_fail((c), _e);  \
    } while (0)

// Order the context's stream after the correlator copies of the last
// qsg_read_correlators_async (they read buffers the next finish, measurement
// or initialisation writes).
static qsg_status order_after_copies(qsg_ctx *c) {
    if (!c->copy_pending) return QSG_OK;
    QSG_CUDA(c, cudaStreamWaitEvent(c->stream, c->copy_ev, 0));
    c->copy_pending = false;
    return QSG_OK;
}

static qsg_status check_device_flag(qsg_ctx *c) {
    int h = 0;
    QSG_CUDA(c, cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    QSG_CUDA(c, cudaStreamSynchronize(c->stream));
    return h == DEVERR_NONE ? QSG_OK : QSG_ERR_TIMEOUT;
}

// Build the persistent-launch plan (all groups with the same algorithm, L <= 24,
// L_tau a multiple of 16) and copy it to the workspace.
static qsg_status upload_plan(qsg_ctx *c) {
    c->plan_ok = false;
    const int ng = (int)c->groups.size();
    for (const Group &g : c->groups)
        if (g.algo != c->groups[0].algo || g.L > 24 || wavefront_chunk(g, c->chunk) == 0) return QSG_OK;
    std::vector<int> order(ng), prefix(ng + 1, 0), chunk(ng);
    for (int i = 0; i < ng; ++i) {
        order[i] = i;
        chunk[i] = wavefront_chunk(c->groups[i], c->chunk);
    }
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        return (double)c->groups[x].nslots * c->groups[x].N > (double)c->groups[y].nslots * c->groups[y].N;
    });
    for (int i = 0; i < ng; ++i) {
        const Group &g = c->groups[order[i]];
        prefix[i + 1] = prefix[i] + g.nslots * (g.Ltau / chunk[order[i]]);
    }
    QSG_CUDA(c, cudaMemcpyAsync(c->pb.groups, c->groups.data(), sizeof(Group) * ng, cudaMemcpyHostToDevice, c->stream));
    QSG_CUDA(c, cudaMemcpyAsync(c->pb.order, order.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, c->stream));
    QSG_CUDA(c, cudaMemcpyAsync(c->pb.prefix, prefix.data(), sizeof(int) * (ng + 1), cudaMemcpyHostToDevice, c->stream));
    QSG_CUDA(c, cudaMemcpyAsync(c->pb.chunk, chunk.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, c->stream));
    QSG_CUDA(c, cudaStreamSynchronize(c->stream));
    c->plan = PersistentPlan{c->pb.groups, c->pb.order, c->pb.prefix, c->pb.chunk, c->pb.queue, ng, prefix[ng],
                             c->groups[0].algo};
    c->plan_ok = true;
    return QSG_OK;
}

extern "C" {

size_t qsg_workspace_bytes(const qsg_shape *shapes, int32_t n_groups) {
    if (!shapes || n_groups < 1 || n_groups > 255) return 0;
    std::vector<Group> gs;
    for (int i = 0; i < n_groups; ++i) {
        if (!valid_shape(shapes[i])) return 0;
        gs.push_back(describe(shapes[i], i));
    }
    int *e;
    uint64_t *s;
    size_t sw;
    return carve(gs, nullptr, &e, &s, &sw);
}

qsg_status qsg_create(qsg_ctx **out, const qsg_shape *shapes, int32_t n_groups, void *d_workspace,
                      size_t workspace_bytes, void *cuda_stream) {
    if (!out || !shapes) return QSG_ERR_ARG;
    *out = nullptr;
    if (n_groups < 1 || n_groups > 255) return QSG_ERR_ARG;
    for (int i = 0; i < n_groups; ++i)
        if (!valid_shape(shapes[i])) return QSG_ERR_SHAPE;
    const size_t need = qsg_workspace_bytes(shapes, n_groups);
    if (!d_workspace || workspace_bytes < need || ((uintptr_t)d_workspace % kAlign) != 0) return QSG_ERR_WORKSPACE;
    qsg_ctx *c = new qsg_ctx();
    c->shapes.assign(shapes, shapes + n_groups);
    for (int i = 0; i < n_groups; ++i) c->groups.push_back(describe(shapes[i], i));
    c->ws = (char *)d_workspace;
    c->ws_bytes = workspace_bytes;
    carve(c->groups, c->ws, &c->d_err, &c->scratch, &c->scratch_words, &c->pb);
    c->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemsetAsync(c->d_err, 0, sizeof(int) * 4, c->stream);
    for (const Group &g : c->groups)
        if (e == cudaSuccess)
            e = cudaMemsetAsync(g.arrivals, 0, sizeof(unsigned) * (size_t)g.nslots * (g.Ltau / 4 > 0 ? g.Ltau / 4 : 1),
                                c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->pb.queue, 0, sizeof(unsigned) * 2, c->stream);
    if (e != cudaSuccess) {
        delete c;
        return QSG_ERR_CUDA;
    }
    *out = c;
    return upload_plan(c);
}

void qsg_destroy(qsg_ctx *ctx) { delete ctx; }

qsg_status qsg_set_stream(qsg_ctx *ctx, void *cuda_stream) {
    if (!ctx) return QSG_ERR_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return QSG_OK;
}

qsg_status qsg_init_samples(qsg_ctx *ctx, uint64_t seed, const double *k_ladders) {
    Range range("qsg_init_samples");
    if (!ctx || !k_ladders) return QSG_ERR_ARG;
    // validate every ladder and build every table before touching the device
    std::vector<std::vector<uint32_t>> thr(ctx->groups.size());
    std::vector<std::vector<uint64_t>> A(ctx->groups.size()), B(ctx->groups.size());
    std::vector<std::vector<int32_t>> Aoff(ctx->groups.size()), Alen(ctx->groups.size());
    std::vector<std::vector<double>> wcos(ctx->groups.size());
    const double *lad = k_ladders;
    for (size_t gi = 0; gi < ctx->groups.size(); ++gi) {
        const Group &g = ctx->groups[gi];
        thr[gi].assign(16 * (size_t)g.K, 0u);
        if (!build_accept_tables(lad, g.K, thr[gi].data())) return QSG_ERR_ARG;
        // cos(2 pi d / L) of the momentum sums of the one-time observables
        for (int d = 0; d <= g.L / 2; ++d) wcos[gi].push_back(std::cos(2.0 * 3.14159265358979323846 * d / g.L));
        const int np = g.K > 1 ? g.K - 1 : 1;
        const long long nmax_blocks = (6LL * g.N >> 6) + 1;
        B[gi].assign(64 * (size_t)np, 0);
        Aoff[gi].assign(np, 0);
        Alen[gi].assign(np, 0);
        for (int i = 0; i + 1 < g.K; ++i) {
            const double delta = lad[i + 1] - lad[i];
            for (int r = 0; r < 64; ++r) B[gi][64 * i + r] = pt_factor(delta, r);
            long long len = 0;
            while (len < nmax_blocks && pt_factor(delta, 64 * len) != 0) ++len;
            if (len > kMaxA) return QSG_ERR_ARG;  // ladder spacing too fine for the table
            Aoff[gi][i] = (int32_t)(i * a_cap(g));
            Alen[gi][i] = (int32_t)len;
            A[gi].resize((size_t)(i + 1) * a_cap(g), 0);
            for (long long m = 0; m < len; ++m) A[gi][(size_t)i * a_cap(g) + m] = pt_factor(delta, 64 * m);
        }
        lad += g.K;
    }
    ctx->seed = seed;
    if (qsg_status o = order_after_copies(ctx)) return o;
    cudaStream_t st = ctx->stream;
    for (size_t gi = 0; gi < ctx->groups.size(); ++gi) {
        const Group &g = ctx->groups[gi];
        const int np = g.K > 1 ? g.K - 1 : 1;
        QSG_CUDA(ctx, cudaMemcpyAsync(g.thr, thr[gi].data(), sizeof(uint32_t) * thr[gi].size(), cudaMemcpyHostToDevice, st));
        if (!A[gi].empty())
            QSG_CUDA(ctx, cudaMemcpyAsync(g.ptA, A[gi].data(), sizeof(uint64_t) * A[gi].size(), cudaMemcpyHostToDevice, st));
        QSG_CUDA(ctx, cudaMemcpyAsync(g.ptB, B[gi].data(), sizeof(uint64_t) * B[gi].size(), cudaMemcpyHostToDevice, st));
        QSG_CUDA(ctx, cudaMemcpyAsync(g.ptA_off, Aoff[gi].data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice, st));
        QSG_CUDA(ctx, cudaMemcpyAsync(g.ptA_len, Alen[gi].data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice, st));
        QSG_CUDA(ctx, launch_init_couplings(g, seed, st));
        QSG_CUDA(ctx, launch_init_spins(g, seed, st));
        const size_t nc = (size_t)g.R * g.W * 64 * g.K * g.nlag;
        QSG_CUDA(ctx, cudaMemsetAsync(g.Cacc, 0, sizeof(long long) * nc, st));
        QSG_CUDA(ctx, cudaMemsetAsync(g.Qacc, 0, sizeof(long long) * nc, st));
        QSG_CUDA(ctx, cudaMemsetAsync(g.Pacc, 0, sizeof(long long) * (size_t)g.W * 64 * g.K, st));
        const size_t nsk = (size_t)g.W * 64 * g.K, nd = (size_t)(g.L / 2 + 1);
        QSG_CUDA(ctx, cudaMemsetAsync(g.P4acc, 0, sizeof(unsigned long long) * 2 * nsk, st));
        QSG_CUDA(ctx, cudaMemsetAsync(g.T3acc, 0, sizeof(long long) * nsk, st));
        QSG_CUDA(ctx, cudaMemsetAsync(g.Gacc, 0, sizeof(long long) * nsk * nd, st));
        QSG_CUDA(ctx, cudaMemsetAsync(g.F3acc, 0, sizeof(long long) * nsk * nd, st));
        QSG_CUDA(ctx, cudaMemsetAsync(g.PPacc, 0, sizeof(long long) * nsk * (size_t)(g.R * (g.R - 1) / 2 + 1), st));
        QSG_CUDA(ctx, cudaMemcpyAsync(g.wcos, wcos[gi].data(), sizeof(double) * nd, cudaMemcpyHostToDevice, st));
        QSG_CUDA(ctx, cudaMemsetAsync(g.acc, 0, sizeof(unsigned long long) * (size_t)g.W * 64 * np, st));
    }
    // host copies of the tables must stay alive until the copies complete
    QSG_CUDA(ctx, cudaStreamSynchronize(st));
    ctx->sweeps = 0;
    ctx->swaps = 0;
    ctx->n_meas = 0;
    ctx->energy_fresh = false;
    ctx->base_valid = false;
    ctx->initialised = true;
    return QSG_OK;
}

qsg_status qsg_set_couplings(qsg_ctx *ctx, int32_t group, const int8_t *J_host) {
    if (!ctx || !J_host || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    const Group &g = ctx->groups[group];
    const int L2 = g.L * g.L;
    std::vector<uint64_t> jx((size_t)g.W * L2, 0), jy((size_t)g.W * L2, 0);
    for (int b = 0; b < g.n_samples; ++b)
        for (int d = 0; d < 2; ++d)
            for (int n = 0; n < L2; ++n) {
                const int8_t v = J_host[((size_t)b * 2 + d) * L2 + n];
                if (v != 1 && v != -1) return QSG_ERR_ARG;
                if (v == -1) (d == 0 ? jx : jy)[(size_t)(b / 64) * L2 + n] |= 1ull << (b % 64);
            }
    QSG_CUDA(ctx, cudaMemcpyAsync(g.Jx, jx.data(), sizeof(uint64_t) * jx.size(), cudaMemcpyHostToDevice, ctx->stream));
    QSG_CUDA(ctx, cudaMemcpyAsync(g.Jy, jy.data(), sizeof(uint64_t) * jy.size(), cudaMemcpyHostToDevice, ctx->stream));
    QSG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->energy_fresh = false;
    return QSG_OK;
}

// Launch one sweep of every group; the sweep index is *sb + idx (sb may be null).
// How the groups of one sweep are launched.
enum SweepMode { MODE_SEQUENTIAL = 0, MODE_PERSISTENT = 1, MODE_CONCURRENT = 2 };

static SweepMode sweep_mode(const qsg_ctx *ctx) {
    if (ctx->sweep_kernel == 1 || ctx->groups.size() < 2) return MODE_SEQUENTIAL;
    if (ctx->persistent == 2 && ctx->plan_ok) return MODE_PERSISTENT;
    if (ctx->persistent == 1) return MODE_SEQUENTIAL;
    return MODE_CONCURRENT;  // 3, or automatic with several groups
}

static qsg_status launch_one_sweep(qsg_ctx *ctx, bool persistent, const uint32_t *sb, uint32_t idx, cudaStream_t st);

// `count` sweeps of every group with indices first .. first + count - 1 (added
// to *sb when sb is given).  Concurrent mode: each group's chain of sweeps on
// its own stream, forked from st and joined back into it (groups share no
// data, so only each group's own sweeps are ordered).
static qsg_status launch_sweeps(qsg_ctx *ctx, SweepMode mode, const uint32_t *sb, uint32_t first, int count,
                                cudaStream_t st) {
    if (mode != MODE_CONCURRENT) {
        for (int i = 0; i < count; ++i) {
            qsg_status s = launch_one_sweep(ctx, mode == MODE_PERSISTENT, sb, first + (uint32_t)i, st);
            if (s != QSG_OK) return s;
        }
        return QSG_OK;
    }
    const size_t ng = ctx->groups.size();
    if (!ctx->fork) QSG_CUDA(ctx, cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming));
    while (ctx->side.size() < ng) {
        cudaStream_t t = nullptr;
        cudaEvent_t e = nullptr;
        QSG_CUDA(ctx, cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
        ctx->side.push_back(t);
        QSG_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->joins.push_back(e);
    }
    QSG_CUDA(ctx, cudaEventRecord(ctx->fork, st));
    for (size_t gi = 0; gi < ng; ++gi) {
        const Group &g = ctx->groups[gi];
        cudaStream_t t = ctx->side[gi];
        QSG_CUDA(ctx, cudaStreamWaitEvent(t, ctx->fork, 0));
        const int C = wavefront_chunk(g, ctx->chunk);
        for (int i = 0; i < count; ++i) {
            if (C > 0)
                QSG_CUDA(ctx, launch_sweep_wavefront(g, sb, first + (uint32_t)i, ctx->seed, g.arrivals, C, ctx->tail, t));
            else if (sb)
                return QSG_ERR_ARG;
            else
                QSG_CUDA(ctx, launch_sweep_reference(g, first + (uint32_t)i, ctx->seed, t));
        }
        QSG_CUDA(ctx, cudaEventRecord(ctx->joins[gi], t));
        QSG_CUDA(ctx, cudaStreamWaitEvent(st, ctx->joins[gi], 0));
    }
    return QSG_OK;
}

static qsg_status launch_one_sweep(qsg_ctx *ctx, bool persistent, const uint32_t *sb, uint32_t idx, cudaStream_t st) {
    if (persistent) {
        QSG_CUDA(ctx, launch_sweep_persistent(ctx->plan, sb, idx, ctx->seed, st));
        return QSG_OK;
    }
    for (const Group &g : ctx->groups) {
        const int C = ctx->sweep_kernel == 1 ? 0 : wavefront_chunk(g, ctx->chunk);
        if (C > 0)
            QSG_CUDA(ctx, launch_sweep_wavefront(g, sb, idx, ctx->seed, g.arrivals, C, ctx->tail, st));
        else if (sb)
            return QSG_ERR_ARG;  // the reference kernel takes its index by value only
        else
            QSG_CUDA(ctx, launch_sweep_reference(g, idx, ctx->seed, st));
    }
    return QSG_OK;
}

// (Re)capture the graph of graph_batch sweeps when a launch option changed.
static qsg_status ensure_graph(qsg_ctx *ctx, SweepMode mode) {
    const long long key = ((((((long long)ctx->graph_batch * 4 + ctx->sweep_kernel) * 4 + (int)mode) * 4 +
                             g_wavefront_variant) * 65537LL + ctx->chunk) * 65537LL + ctx->tail) * 32 + ctx->upb;
    if (ctx->graph_exec && ctx->graph_key == key) return QSG_OK;
    if (ctx->graph_exec) {
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
    }
    if (!ctx->cap_stream) QSG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    const unsigned long long before = g_launches.load();
    QSG_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed));
    qsg_status s = launch_sweeps(ctx, mode, ctx->pb.sweep_base, 0u, ctx->graph_batch, ctx->cap_stream);
    if (s == QSG_OK && launch_add_word(ctx->pb.sweep_base, (uint32_t)ctx->graph_batch, ctx->cap_stream) != cudaSuccess)
        s = QSG_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(ctx->cap_stream, &graph);
    const unsigned long long captured = g_launches.load() - before;
    g_launches.fetch_sub(captured);  // captured launches run only when replayed
    if (s != QSG_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e_end != cudaSuccess) return cuda_fail(ctx, e_end);
    const cudaError_t e_inst = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e_inst != cudaSuccess) {
        ctx->graph_exec = nullptr;
        return cuda_fail(ctx, e_inst);
    }
    ctx->graph_key = key;
    ctx->graph_launches = captured;
    return QSG_OK;
}

qsg_status qsg_sweep(qsg_ctx *ctx, int32_t n_sweeps) {
    Range range("qsg_sweep");
    if (!ctx || n_sweeps < 0) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    if ((uint64_t)ctx->sweeps + (uint64_t)n_sweeps > 0xFFFFFFFFull) return QSG_ERR_ARG;
    const SweepMode mode = sweep_mode(ctx);
    int done = 0;
    const int G = ctx->graph_batch;
    if (G > 0 && n_sweeps >= G) {
        qsg_status s = ensure_graph(ctx, mode);
        if (s != QSG_OK) return s;
        if (!ctx->base_valid) {
            QSG_CUDA(ctx, launch_set_word(ctx->pb.sweep_base, ctx->sweeps, ctx->stream));
            ctx->base_valid = true;
        }
        for (; done + G <= n_sweeps; done += G) {
            QSG_CUDA(ctx, cudaGraphLaunch(ctx->graph_exec, ctx->stream));
            count_launches((int)ctx->graph_launches);
            ctx->sweeps += (uint32_t)G;
        }
    }
    if (done < n_sweeps) {
        qsg_status s = launch_sweeps(ctx, mode, nullptr, ctx->sweeps, n_sweeps - done, ctx->stream);
        if (s != QSG_OK) return s;
        ctx->sweeps += (uint32_t)(n_sweeps - done);
        ctx->base_valid = false;
    }
    if (n_sweeps > 0) ctx->energy_fresh = false;
    return QSG_OK;
}

static qsg_status ensure_energy(qsg_ctx *ctx) {
    if (ctx->energy_fresh) return QSG_OK;
    for (const Group &g : ctx->groups) QSG_CUDA(ctx, launch_energy(g, ctx->stream));
    ctx->energy_fresh = true;
    return QSG_OK;
}

qsg_status qsg_tempering_swap(qsg_ctx *ctx) {
    Range range("qsg_tempering_swap");
    if (!ctx) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    qsg_status s = ensure_energy(ctx);
    if (s != QSG_OK) return s;
    for (const Group &g : ctx->groups) QSG_CUDA(ctx, launch_tempering(g, ctx->swaps, ctx->seed, ctx->stream));
    ctx->swaps++;
    return QSG_OK;
}

qsg_status qsg_measure_correlators(qsg_ctx *ctx) {
    Range range("qsg_measure_correlators");
    if (!ctx) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    if (qsg_status o = order_after_copies(ctx)) return o;
    for (const Group &g : ctx->groups)
        QSG_CUDA(ctx, launch_measure(g, ctx->scratch, ctx->scratch_words, ctx->corr_tensor, ctx->triples, ctx->d_err,
                                     ctx->wait_limit, ctx->stream));
    ctx->n_meas++;
    return QSG_OK;
}

// The copies of qsg_read_correlators on stream st.
static qsg_status copy_correlators(qsg_ctx *ctx, const Group &g, double *C, double *Q2, double *q2, int64_t *raw,
                                   cudaStream_t st) {
    // device layout [R][W*64][K][nl]; the host keeps the first n_samples of the
    // W*64 sample bits, so every replica is one contiguous block on both sides
    // and the copies go straight into the caller's buffers (at DMA speed when
    // they are page-locked)
    const int S = g.n_samples, Sp = g.W * 64, K = g.K, nl = g.nlag;
    const size_t blk = (size_t)S * K * nl, pitch = (size_t)Sp * K * nl, outc = (size_t)g.R * blk;
    for (int r = 0; r < g.R; ++r) {
        if (C)
            QSG_CUDA(ctx, cudaMemcpyAsync(C + r * blk, g.outC + r * pitch, sizeof(double) * blk, cudaMemcpyDeviceToHost, st));
        if (Q2)
            QSG_CUDA(ctx, cudaMemcpyAsync(Q2 + r * blk, g.outQ + r * pitch, sizeof(double) * blk, cudaMemcpyDeviceToHost, st));
        if (raw) {
            QSG_CUDA(ctx, cudaMemcpyAsync(raw + r * blk, g.Cacc + r * pitch, sizeof(long long) * blk,
                                          cudaMemcpyDeviceToHost, st));
            QSG_CUDA(ctx, cudaMemcpyAsync(raw + outc + r * blk, g.Qacc + r * pitch, sizeof(long long) * blk,
                                          cudaMemcpyDeviceToHost, st));
        }
    }
    if (q2) QSG_CUDA(ctx, cudaMemcpyAsync(q2, g.outP, sizeof(double) * (size_t)S * K, cudaMemcpyDeviceToHost, st));
    if (raw)
        QSG_CUDA(ctx, cudaMemcpyAsync(raw + 2 * outc, g.Pacc, sizeof(long long) * (size_t)S * K, cudaMemcpyDeviceToHost,
                                      st));
    return QSG_OK;
}

qsg_status qsg_read_correlators(qsg_ctx *ctx, int32_t group, double *C, double *Q2, double *q2, int64_t *raw) {
    Range range("qsg_read_correlators");
    if (!ctx || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    if (qsg_status o = order_after_copies(ctx)) return o;
    const Group &g = ctx->groups[group];
    QSG_CUDA(ctx, launch_finish(g, ctx->n_meas, ctx->stream));
    if (qsg_status o = copy_correlators(ctx, g, C, Q2, q2, raw, ctx->stream)) return o;
    return check_device_flag(ctx);
}

qsg_status qsg_read_correlators_async(qsg_ctx *ctx, int32_t group, double *C, double *Q2, double *q2, int64_t *raw,
                                      void *copy_stream) {
    Range range("qsg_read_correlators_async");
    if (!ctx || !copy_stream || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    cudaStream_t cs = static_cast<cudaStream_t>(copy_stream);
    if (cs == ctx->stream) return QSG_ERR_ARG;
    if (qsg_status o = order_after_copies(ctx)) return o;
    if (!ctx->fin_ev) QSG_CUDA(ctx, cudaEventCreateWithFlags(&ctx->fin_ev, cudaEventDisableTiming));
    if (!ctx->copy_ev) QSG_CUDA(ctx, cudaEventCreateWithFlags(&ctx->copy_ev, cudaEventDisableTiming));
    if (!ctx->h_flag) QSG_CUDA(ctx, cudaHostAlloc((void **)&ctx->h_flag, sizeof(int), cudaHostAllocDefault));
    const Group &g = ctx->groups[group];
    // the finish runs on the copy stream too, once the context's stream has
    // done the measurements: it writes only what the copies read, and the
    // next writer of the sums waits for the copies
    QSG_CUDA(ctx, cudaEventRecord(ctx->fin_ev, ctx->stream));
    QSG_CUDA(ctx, cudaStreamWaitEvent(cs, ctx->fin_ev, 0));
    QSG_CUDA(ctx, launch_finish(g, ctx->n_meas, cs));
    if (qsg_status o = copy_correlators(ctx, g, C, Q2, q2, raw, cs)) return o;
    QSG_CUDA(ctx, cudaMemcpyAsync(ctx->h_flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, cs));
    QSG_CUDA(ctx, cudaEventRecord(ctx->copy_ev, cs));
    ctx->copy_pending = true;
    ctx->flag_pending = true;
    return QSG_OK;
}

qsg_status qsg_wait_correlators(qsg_ctx *ctx) {
    if (!ctx) return QSG_ERR_ARG;
    if (!ctx->flag_pending) return QSG_OK;
    QSG_CUDA(ctx, cudaEventSynchronize(ctx->copy_ev));
    ctx->flag_pending = false;
    return *ctx->h_flag == DEVERR_NONE ? QSG_OK : QSG_ERR_TIMEOUT;
}

qsg_status qsg_read_onetime(qsg_ctx *ctx, int32_t group, double *per_sample, double *per_k, int64_t *raw) {
    if (!ctx || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    const Group &g = ctx->groups[group];
    const size_t nsk = (size_t)g.W * 64 * g.K, nd = (size_t)(g.L / 2 + 1);
    QSG_CUDA(ctx, launch_onetime_finish(g, ctx->n_meas, ctx->triples, ctx->stream));
    std::vector<double> ho(nsk * 7), hk((size_t)g.K * 8);
    std::vector<long long> rp, rt, rg, rf;
    std::vector<unsigned long long> r4;
    QSG_CUDA(ctx, cudaMemcpyAsync(ho.data(), g.outO, sizeof(double) * ho.size(), cudaMemcpyDeviceToHost, ctx->stream));
    QSG_CUDA(ctx, cudaMemcpyAsync(hk.data(), g.outK, sizeof(double) * hk.size(), cudaMemcpyDeviceToHost, ctx->stream));
    if (raw) {
        rp.resize(nsk);
        rt.resize(nsk);
        r4.resize(2 * nsk);
        rg.resize(nsk * nd);
        rf.resize(nsk * nd);
        QSG_CUDA(ctx, cudaMemcpyAsync(rp.data(), g.Pacc, sizeof(long long) * nsk, cudaMemcpyDeviceToHost, ctx->stream));
        QSG_CUDA(ctx, cudaMemcpyAsync(rt.data(), g.T3acc, sizeof(long long) * nsk, cudaMemcpyDeviceToHost, ctx->stream));
        QSG_CUDA(ctx, cudaMemcpyAsync(r4.data(), g.P4acc, sizeof(unsigned long long) * 2 * nsk, cudaMemcpyDeviceToHost,
                                      ctx->stream));
        QSG_CUDA(ctx, cudaMemcpyAsync(rg.data(), g.Gacc, sizeof(long long) * nsk * nd, cudaMemcpyDeviceToHost,
                                      ctx->stream));
        QSG_CUDA(ctx, cudaMemcpyAsync(rf.data(), g.F3acc, sizeof(long long) * nsk * nd, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    }
    QSG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const size_t ns = (size_t)g.n_samples * g.K;
    if (per_sample) std::memcpy(per_sample, ho.data(), sizeof(double) * ns * 7);
    if (per_k) std::memcpy(per_k, hk.data(), sizeof(double) * hk.size());
    if (raw) {
        const size_t rw = 4 + 2 * nd;
        for (size_t c = 0; c < ns; ++c) {
            int64_t *o = raw + c * rw;
            // sum of Q^4 = high part * 2^32 + low part, as a 128-bit integer
            const unsigned __int128 p4 = ((unsigned __int128)r4[2 * c + 1] << 32) + (unsigned __int128)r4[2 * c];
            o[0] = rp[c];
            o[1] = (int64_t)(uint64_t)p4;
            o[2] = (int64_t)(uint64_t)(p4 >> 64);
            o[3] = rt[c];
            for (size_t d = 0; d < nd; ++d) {
                o[4 + d] = rg[c * nd + d];
                o[4 + nd + d] = rf[c * nd + d];
            }
        }
    }
    return QSG_OK;
}

qsg_status qsg_read_pair_overlaps(qsg_ctx *ctx, int32_t group, int64_t *out) {
    if (!ctx || !out || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    const Group &g = ctx->groups[group];
    const size_t np = (size_t)(g.R * (g.R - 1) / 2);
    if (np == 0) return QSG_OK;
    QSG_CUDA(ctx, cudaMemcpyAsync(out, g.PPacc, sizeof(long long) * (size_t)g.n_samples * g.K * np,
                                  cudaMemcpyDeviceToHost, ctx->stream));
    QSG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return QSG_OK;
}

qsg_status qsg_sample_features(qsg_ctx *ctx, int32_t group, float *out) {
    if (!ctx || !out || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    const Group &g = ctx->groups[group];
    // the correlator scratch is free between calls: it holds the features
    if (ctx->scratch_words * sizeof(uint64_t) < (size_t)g.W * 64 * 64 * sizeof(float)) return QSG_ERR_WORKSPACE;
    float *d = reinterpret_cast<float *>(ctx->scratch);
    QSG_CUDA(ctx, launch_features(g, d, ctx->stream));
    QSG_CUDA(ctx, cudaMemcpyAsync(out, d, sizeof(float) * (size_t)g.n_samples * 64, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    QSG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return QSG_OK;
}

qsg_status qsg_read_energies(qsg_ctx *ctx, int32_t group, int64_t *E_host) {
    if (!ctx || !E_host || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    qsg_status s = ensure_energy(ctx);
    if (s != QSG_OK) return s;
    const Group &g = ctx->groups[group];
    std::vector<int32_t> U((size_t)g.nslots * 64);
    QSG_CUDA(ctx, cudaMemcpyAsync(U.data(), g.U, sizeof(int32_t) * U.size(), cudaMemcpyDeviceToHost, ctx->stream));
    QSG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int b = 0; b < g.n_samples; ++b)
        for (int r = 0; r < g.R; ++r)
            for (int j = 0; j < g.K; ++j) {
                const size_t slot = ((size_t)(b / 64) * g.R + r) * g.K + j;
                E_host[((size_t)b * g.R + r) * g.K + j] = 2LL * U[slot * 64 + (b % 64)] - 3LL * g.N;
            }
    return QSG_OK;
}

qsg_status qsg_read_accepts(qsg_ctx *ctx, int32_t group, int64_t *acc_host) {
    if (!ctx || !acc_host || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    const Group &g = ctx->groups[group];
    const int np = g.K > 1 ? g.K - 1 : 1;
    std::vector<unsigned long long> a((size_t)g.W * 64 * np);
    QSG_CUDA(ctx, cudaMemcpyAsync(a.data(), g.acc, sizeof(unsigned long long) * a.size(), cudaMemcpyDeviceToHost, ctx->stream));
    QSG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < (size_t)g.n_samples * np; ++i) acc_host[i] = (int64_t)a[i];
    return QSG_OK;
}

qsg_status qsg_get_spins(qsg_ctx *ctx, int32_t group, uint64_t *host) {
    if (!ctx || !host || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    const Group &g = ctx->groups[group];
    QSG_CUDA(ctx, cudaMemcpyAsync(host, g.S, sizeof(uint64_t) * (size_t)g.nslots * g.N, cudaMemcpyDeviceToHost, ctx->stream));
    QSG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return QSG_OK;
}

qsg_status qsg_set_spins(qsg_ctx *ctx, int32_t group, const uint64_t *host) {
    if (!ctx || !host || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    const Group &g = ctx->groups[group];
    QSG_CUDA(ctx, cudaMemcpyAsync(g.S, host, sizeof(uint64_t) * (size_t)g.nslots * g.N, cudaMemcpyHostToDevice, ctx->stream));
    QSG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->energy_fresh = false;
    return QSG_OK;
}

qsg_status qsg_get_spins_device(qsg_ctx *ctx, int32_t group, uint64_t *d_out) {
    if (!ctx || !d_out || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    const Group &g = ctx->groups[group];
    QSG_CUDA(ctx, launch_copy_words(d_out, g.S, (size_t)g.nslots * g.N, ctx->stream));
    return QSG_OK;
}

qsg_status qsg_set_spins_device(qsg_ctx *ctx, int32_t group, const uint64_t *d_words) {
    if (!ctx || !d_words || group < 0 || group >= (int)ctx->groups.size()) return QSG_ERR_ARG;
    const Group &g = ctx->groups[group];
    QSG_CUDA(ctx, launch_copy_words(g.S, d_words, (size_t)g.nslots * g.N, ctx->stream));
    ctx->energy_fresh = false;
    return QSG_OK;
}

qsg_status qsg_get_counters(qsg_ctx *ctx, uint32_t *sweeps, uint32_t *swaps, int64_t *n_meas) {
    if (!ctx) return QSG_ERR_ARG;
    if (sweeps) *sweeps = ctx->sweeps;
    if (swaps) *swaps = ctx->swaps;
    if (n_meas) *n_meas = ctx->n_meas;
    return QSG_OK;
}

qsg_status qsg_set_counters(qsg_ctx *ctx, uint32_t sweeps, uint32_t swaps, int64_t n_meas) {
    if (!ctx) return QSG_ERR_ARG;
    if (!ctx->initialised) return QSG_ERR_STATE;
    ctx->sweeps = sweeps;
    ctx->base_valid = false;
    ctx->swaps = swaps;
    if (n_meas >= 0) ctx->n_meas = n_meas;
    return QSG_OK;
}

qsg_status qsg_set_option(qsg_ctx *ctx, int32_t option, int64_t value) {
    if (!ctx) return QSG_ERR_ARG;
    if (option == QSG_OPT_SWEEP_KERNEL) {
        if (value < 0 || value > 2) return QSG_ERR_ARG;
        if (value == 2)
            for (const Group &g : ctx->groups)
                if (wavefront_chunk(g, ctx->chunk) == 0) return QSG_ERR_ARG;
        if (value == 1 && ctx->graph_batch > 0) return QSG_ERR_ARG;
        ctx->sweep_kernel = (int)value;
        return QSG_OK;
    }
    if (option == QSG_OPT_WAVEFRONT_VARIANT) {
        if (value < 0 || value > 3) return QSG_ERR_ARG;
        g_wavefront_variant = (int)value;
        return QSG_OK;
    }
    if (option == QSG_OPT_PERSISTENT) {
        if (value < 0 || value > 3) return QSG_ERR_ARG;
        if (value == 2 && !ctx->plan_ok) return QSG_ERR_ARG;
        ctx->persistent = (int)value;
        return QSG_OK;
    }
    if (option == QSG_OPT_GRAPH) {
        if (value < 0 || value > 4096) return QSG_ERR_ARG;
        if (value > 0 && ctx->sweep_kernel == 1) return QSG_ERR_ARG;
        if (value > 0)
            for (const Group &g : ctx->groups)
                if (wavefront_chunk(g, ctx->chunk) == 0) return QSG_ERR_ARG;
        ctx->graph_batch = (int)value;
        return QSG_OK;
    }
    if (option == QSG_OPT_ONETIME) {
        if (value < 0 || value > 1) return QSG_ERR_ARG;
        // the three-replica sums accumulate only while enabled: changing it
        // between measurements would mix counts, so it must precede the first
        if (ctx->n_meas > 0 && (value == 0) != (ctx->triples == 1)) return QSG_ERR_STATE;
        ctx->triples = value == 0 ? 1 : 0;
        return QSG_OK;
    }
    if (option == QSG_OPT_CORR_KERNEL) {
        if (value < 0 || value > 1) return QSG_ERR_ARG;
        ctx->corr_tensor = value == 0 ? 1 : 0;
        return QSG_OK;
    }
    if (option == QSG_OPT_TAIL) {
        if (value < 0 || value > (1 << 24)) return QSG_ERR_ARG;
        ctx->tail = (int)value;
        return QSG_OK;
    }
    if (option == QSG_OPT_UNITS_PER_BLOCK) {
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16) return QSG_ERR_ARG;
        ctx->upb = (int)value;
        for (Group &g : ctx->groups) g.upb = ctx->upb;
        return QSG_OK;
    }
    if (option == QSG_OPT_WAIT_LIMIT) {
        if (value < 0 || value > (1LL << 30)) return QSG_ERR_ARG;
        ctx->wait_limit = (unsigned)value;
        return QSG_OK;
    }
    if (option == QSG_OPT_CHUNK) {
        if (value < 0 || value > 65536) return QSG_ERR_ARG;
        if (value > 0 || ctx->graph_batch > 0)
            for (const Group &g : ctx->groups)
                if (wavefront_chunk(g, (int)value) == 0) return QSG_ERR_ARG;
        ctx->chunk = (int)value;
        return upload_plan(ctx);
    }
    return QSG_ERR_ARG;
}

uint64_t qsg_kernel_launches(void) { return (uint64_t)g_launches.load(); }

const char *qsg_strerror(qsg_status status) {
    switch (status) {
        case QSG_OK: return "ok";
        case QSG_ERR_ARG: return "invalid argument";
        case QSG_ERR_SHAPE: return "invalid group shape";
        case QSG_ERR_CUDA: return "CUDA runtime error";
        case QSG_ERR_TIMEOUT: return "bounded device wait gave up";
        case QSG_ERR_STATE: return "call out of order";
        case QSG_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    }
    return "unknown status";
}

const char *qsg_last_cuda_error(qsg_ctx *ctx) { return ctx ? ctx->last_cuda.c_str() : ""; }

}  // extern "C"
