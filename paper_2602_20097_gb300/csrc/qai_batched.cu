// qai_batched.cu -- many fields in one call (see include/qai.h).
//
// Fields are grouped by rank (after squeezing). Rank-2 and rank-3 fields run
// their own plain launch sequence (qai_mitigate without per-step outputs:
// the local first EDT and the signed-point route), dealt round robin onto a
// few streams forked from the caller's, so the small fields' short, latency-
// bound kernels overlap; rank-1 fields run as two grouped row-pass kernels
// over all of them (a CTA finds its field in a table passed by value in the
// kernel parameters). The whole launch sequence of a batch is captured once
// into a CUDA graph and replayed, so a repeated batch costs one graph launch.
// Per group, the stream count and the field order (as given, or largest
// first) come from an autotuner that times the candidates on the batch itself
// and caches the winner by the group's shape signature.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "qai.h"
#include "qai_host.h"
#include "qai_launch.h"

using namespace qai;
using namespace qai::host;

namespace {

struct GroupCfg {
    int order = 1;    // 0: as given, 1: largest field first
    int streams = 4;  // rank 2 and 3: streams the fields' launch sequences are dealt onto
};
constexpr int kMaxStreams = 8;

// Streams forked from a caller's stream (an event recorded there, waited on
// by each) and joined back (one event per stream, waited on by the caller's
// stream). Works inside a stream capture: the forked streams join it.
struct Forker {
    cudaStream_t s[kMaxStreams] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kMaxStreams] = {};
    bool ok = false;
};
Forker* forker()
{
    thread_local Forker f;
    if (!f.ok) {
        bool good = cudaEventCreateWithFlags(&f.fork_ev, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; good && i < kMaxStreams; ++i)
            good = cudaStreamCreateWithFlags(&f.s[i], cudaStreamNonBlocking) == cudaSuccess &&
                   cudaEventCreateWithFlags(&f.join_ev[i], cudaEventDisableTiming) == cudaSuccess;
        if (!good) return nullptr;
        f.ok = true;
    }
    return &f;
}

struct Field {
    int index;
    Shape sh;
    Layout lay;
    size_t ws_off;
    const int32_t* q;
    float* out;
    MethodArgs m;
};

struct Batch {
    std::vector<Field> f;
    std::vector<int> group[4];  // field positions per rank
    size_t ws_total = 0;
};

std::mutex g_mu;
std::unordered_map<uint64_t, GroupCfg> g_tuned;  // group signature -> config
struct GraphEntry {
    uint64_t key;
    cudaGraphExec_t exec;
    int kernels;
};
std::vector<GraphEntry> g_graphs;  // most recent last
constexpr size_t kMaxGraphs = 16;

uint64_t fnv(const void* p, size_t n, uint64_t h)
{
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

uint64_t group_signature(const Batch& bt, int rank)
{
    std::vector<int64_t> v;
    for (int i : bt.group[rank]) {
        v.push_back(bt.f[i].sh.nz);
        v.push_back(bt.f[i].sh.ny);
        v.push_back(bt.f[i].sh.nx);
    }
    std::sort(v.begin(), v.end());
    uint64_t h = fnv(&rank, sizeof rank, 1469598103934665603ull);
    return fnv(v.data(), v.size() * sizeof(int64_t), h);
}

GroupCfg tuned_cfg(uint64_t sig)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_tuned.find(sig);
    return it == g_tuned.end() ? GroupCfg() : it->second;
}

qai_status plan(int n, const int32_t* const* d_q, float* const* d_out, const int32_t* ranks,
                const int64_t* dims, const double* eb, const qai_params* params, Batch& bt)
{
    if (n < 1) return fail(QAI_ERR_INVALID_ARG, "n must be >= 1");
    if (!d_q || !d_out || !ranks || !dims || !eb) return fail(QAI_ERR_INVALID_ARG, "NULL array argument");
    qai_params defaults;
    qai_default_params(&defaults);
    const qai_params* p = params ? params : &defaults;
    qai_status s = check_params(p);
    if (s != QAI_OK) return s;
    bt.f.resize(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        Field& f = bt.f[i];
        f.index = i;
        if ((s = make_shape(ranks[i], dims + 3 * i, &f.sh)) != QAI_OK) return s;
        if (!d_q[i] || !d_out[i]) return fail(QAI_ERR_INVALID_ARG, "field %d: NULL buffer", i);
        if (!(eb[i] > 0.0) || !std::isfinite(eb[i])) return fail(QAI_ERR_INVALID_ARG, "field %d: bad eb", i);
        f.lay = layout_for(f.sh, 0);
        f.ws_off = off;
        off = align256(off + f.lay.total);
        f.q = d_q[i];
        f.out = d_out[i];
        f.m = method_args(p, eb[i]);
        bt.group[f.sh.rank].push_back(i);
    }
    bt.ws_total = off;
    return QAI_OK;
}

// Rank-1 fields: the grouped row passes (phase 1 writes Dist1 and S, phase 2
// GetBoundary(S), the EDT of B2 and step E), at most kMaxGroup fields a launch.
qai_status launch_rank1(const Batch& bt, const std::vector<int>& order, char* ws, cudaStream_t st, int* kernels)
{
    for (size_t c0 = 0; c0 < order.size(); c0 += kMaxGroup) {
        const int cn = (int)std::min(order.size() - c0, (size_t)kMaxGroup);
        auto F = [&](int k) -> const Field& { return bt.f[order[c0 + k]]; };
        int max_nx = 0;
        for (int k = 0; k < cn; ++k) max_nx = std::max(max_nx, F(k).sh.nx);
        for (int phase = 1; phase <= 2; ++phase) {
            thread_local RowTable rt;  // large: built on the host, copied into the launch
            std::memset(&rt, 0, sizeof rt);
            rt.n = cn;
            rt.smem_nx = max_nx;
            rt.warps = rowpass_warps(max_nx);
            int acc = 0;
            for (int k = 0; k < cn; ++k) {
                const Field& f = F(k);
                char* b = ws + f.ws_off;
                RowArgs r{};
                r.rank = 1; r.nz = f.sh.nz; r.ny = f.sh.ny; r.nx = f.sh.nx;
                r.q = f.q; r.eqm = reinterpret_cast<uint8_t*>(b + f.lay.eqm); r.m = f.m;
                int32_t* dist1 = reinterpret_cast<int32_t*>(b + f.lay.dist1);
                int8_t* s = reinterpret_cast<int8_t*>(b + f.lay.s);
                if (phase == 1) {
                    r.dist1 = dist1; r.s_out = s;
                } else {
                    r.s_in = s; r.dist1_in = dist1; r.out = f.out;
                }
                prepare_rowpass(r);
                rt.args[k] = r;
                rt.first_row[k] = acc;
                acc += f.sh.nz * f.sh.ny;
            }
            rt.first_row[cn] = acc;
            cudaError_t e = launch_rowpass_grouped(phase, true, rt, st);
            ++*kernels;
            if (e != cudaSuccess) return cuda_fail(e, "grouped row pass");
        }
    }
    return QAI_OK;
}

// The launches of one rank group on `st` (rank 2 and 3: on cfg.streams
// streams forked from it and joined back). Adds the kernels launched to
// *kernels.
qai_status launch_group(const Batch& bt, int rank, const GroupCfg& cfg, char* ws, cudaStream_t st,
                        int* kernels)
{
    std::vector<int> order = bt.group[rank];
    if (order.empty()) return QAI_OK;
    if (cfg.order == 1)
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return bt.f[a].sh.N > bt.f[b].sh.N; });
    if (rank == 1) return launch_rank1(bt, order, ws, st, kernels);
    const int ns = std::max(1, std::min(cfg.streams, kMaxStreams));
    Forker* fk = ns > 1 ? forker() : nullptr;
    if (ns > 1 && !fk) return cuda_fail(cudaGetLastError(), "batch streams");
    cudaError_t e;
    if (fk) {
        if ((e = cudaEventRecord(fk->fork_ev, st)) != cudaSuccess) return cuda_fail(e, "fork");
        for (int i = 0; i < ns; ++i)
            if ((e = cudaStreamWaitEvent(fk->s[i], fk->fork_ev, 0)) != cudaSuccess) return cuda_fail(e, "fork");
    }
    qai_status s = QAI_OK;
    {
        LaunchSink sink(kernels);
        for (size_t k = 0; k < order.size() && s == QAI_OK; ++k) {
            const Field& f = bt.f[order[k]];
            s = run_plain(f.q, f.out, f.sh, f.m, ws + f.ws_off, f.lay, fk ? fk->s[k % ns] : st);
        }
    }
    if (fk) {  // join, also after an error, so no stream is left forked
        for (int i = 0; i < ns; ++i) {
            if ((e = cudaEventRecord(fk->join_ev[i], fk->s[i])) != cudaSuccess && s == QAI_OK) s = cuda_fail(e, "join");
            if ((e = cudaStreamWaitEvent(st, fk->join_ev[i], 0)) != cudaSuccess && s == QAI_OK) s = cuda_fail(e, "join");
        }
    }
    return s;
}

qai_status launch_all(const Batch& bt, const GroupCfg cfgs[4], char* ws, cudaStream_t st, int* kernels)
{
    for (int rank = 3; rank >= 1; --rank) {
        qai_status s = launch_group(bt, rank, cfgs[rank], ws, st, kernels);
        if (s != QAI_OK) return s;
    }
    return QAI_OK;
}

qai_status check_ws(const Batch& bt, void* d_ws, size_t ws_bytes)
{
    if (!d_ws) return fail(QAI_ERR_INVALID_ARG, "d_ws must be non-NULL");
    if (ws_bytes < bt.ws_total)
        return fail(QAI_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", ws_bytes, bt.ws_total);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255) return fail(QAI_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    return QAI_OK;
}

}  // namespace

extern "C" {

qai_status qai_workspace_size_batched(int n, const int32_t* ranks, const int64_t* dims, size_t* bytes)
{
    if (!bytes || !ranks || !dims || n < 1) return fail(QAI_ERR_INVALID_ARG, "bad arguments");
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        Shape sh;
        qai_status s = make_shape(ranks[i], dims + 3 * i, &sh);
        if (s != QAI_OK) return s;
        off = align256(off + layout_for(sh, 0).total);
    }
    *bytes = off;
    return QAI_OK;
}

qai_status qai_mitigate_batched(int n, const int32_t* const* d_q, float* const* d_out, const int32_t* ranks,
                                const int64_t* dims, const double* eb, const qai_params* params, void* d_ws,
                                size_t ws_bytes, cudaStream_t stream)
{
    qai::set_last_error("");
    Batch bt;
    qai_status s = plan(n, d_q, d_out, ranks, dims, eb, params, bt);
    if (s != QAI_OK) return s;
    if ((s = check_ws(bt, d_ws, ws_bytes)) != QAI_OK) return s;
    GroupCfg cfgs[4];
    for (int r = 1; r <= 3; ++r) cfgs[r] = tuned_cfg(group_signature(bt, r));
    char* ws = static_cast<char*>(d_ws);

    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return cuda_fail(cudaGetLastError(), "stream query");
    int kernels = 0;
    if (cs != cudaStreamCaptureStatusNone) {  // the caller captures: record the launches into its graph
        s = launch_all(bt, cfgs, ws, stream, &kernels);
        for (int k = 0; k < kernels; ++k) count_launch();
        return s;
    }
    // key of the cached graph: every argument that reaches a kernel
    uint64_t key = fnv(&n, sizeof n, 1469598103934665603ull);
    key = fnv(d_q, n * sizeof(void*), key);
    key = fnv(d_out, n * sizeof(void*), key);
    key = fnv(ranks, n * sizeof(int32_t), key);
    key = fnv(dims, 3 * n * sizeof(int64_t), key);
    key = fnv(eb, n * sizeof(double), key);
    qai_params pv;
    if (params) pv = *params; else qai_default_params(&pv);
    key = fnv(&pv, sizeof pv, key);
    key = fnv(&d_ws, sizeof d_ws, key);
    key = fnv(cfgs, sizeof cfgs, key);
    key = fnv(&stream, sizeof stream, key);

    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (size_t i = 0; i < g_graphs.size(); ++i) {
            if (g_graphs[i].key == key) {
                GraphEntry e = g_graphs[i];
                g_graphs.erase(g_graphs.begin() + i);
                g_graphs.push_back(e);
                exec = e.exec;
                kernels = e.kernels;
                break;
            }
        }
    }
    if (!exec) {
        // Capture on a private stream (the caller's may be the legacy default
        // stream, which cannot capture); the graph is launched on `stream`.
        thread_local cudaStream_t cap = nullptr;
        if (!cap) {
            cudaError_t ec = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            if (ec != cudaSuccess) { cap = nullptr; return cuda_fail(ec, "capture stream"); }
        }
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "begin capture");
        s = launch_all(bt, cfgs, ws, cap, &kernels);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (s != QAI_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_graphs.size() >= kMaxGraphs) {
            cudaGraphExecDestroy(g_graphs.front().exec);
            g_graphs.erase(g_graphs.begin());
        }
        g_graphs.push_back({key, exec, kernels});
    }
    cudaError_t e = cudaGraphLaunch(exec, stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    for (int k = 0; k < kernels; ++k) count_launch();
    return QAI_OK;
}

qai_status qai_autotune_batched(int n, const int32_t* const* d_q, float* const* d_out, const int32_t* ranks,
                                const int64_t* dims, const double* eb, const qai_params* params, void* d_ws,
                                size_t ws_bytes, cudaStream_t stream, qai_batch_choice* choices)
{
    qai::set_last_error("");
    Batch bt;
    qai_status s = plan(n, d_q, d_out, ranks, dims, eb, params, bt);
    if (s != QAI_OK) return s;
    if ((s = check_ws(bt, d_ws, ws_bytes)) != QAI_OK) return s;
    char* ws = static_cast<char*>(d_ws);
    static const GroupCfg cands[] = {{1, 1}, {1, 2}, {1, 4}, {1, 8}, {0, 1}, {0, 2}, {0, 4}, {0, 8}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "event create");
    for (int rank = 1; rank <= 3; ++rank) {
        if (choices) std::memset(&choices[rank - 1], 0, sizeof(qai_batch_choice));
        if (bt.group[rank].empty()) continue;
        float best_ms = 1e30f;
        GroupCfg best;
        for (const GroupCfg& c : cands) {
            if (rank == 1 && c.streams != 1) continue;  // rank 1: one grouped launch per phase
            int kernels = 0;
            if ((s = launch_group(bt, rank, c, ws, stream, &kernels)) != QAI_OK) break;  // warm-up
            cudaEventRecord(e0, stream);
            for (int rep = 0; rep < 3 && s == QAI_OK; ++rep) s = launch_group(bt, rank, c, ws, stream, &kernels);
            cudaEventRecord(e1, stream);
            if (s != QAI_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { s = cuda_fail(cudaGetLastError(), "autotune sync"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3.f;
            if (ms < best_ms) { best_ms = ms; best = c; }
        }
        if (s != QAI_OK) break;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            g_tuned[group_signature(bt, rank)] = best;
        }
        if (choices) {
            qai_batch_choice& ch = choices[rank - 1];
            ch.rank = rank;
            ch.fields = (int32_t)bt.group[rank].size();
            ch.streams = best.streams;
            ch.order = best.order;
            ch.ms = best_ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

}  // extern "C"
