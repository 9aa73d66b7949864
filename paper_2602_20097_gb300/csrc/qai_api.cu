// qai_api.cu -- the C ABI of libqai (see include/qai.h): argument checks,
// workspace layout and the stream-ordered launch sequence of Algorithm 4.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "qai.h"
#include "qai_device.cuh"
#include "qai_host.h"
#include "qai_launch.h"

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace qai {
namespace host {

qai_status fail(qai_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1); }

}  // namespace host
}  // namespace qai

namespace {
using namespace qai::host;

// ---- per-kernel timing ------------------------------------------------------
struct Pending {
    const char* name;
    double bytes;
    cudaEvent_t a, b;
};
struct Stat {
    std::string name;
    int64_t launches = 0;
    double ms = 0, bytes = 0;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
thread_local int* g_launch_sink = nullptr;  // set: count launches here, no events
std::string g_prof_only;  // time only kernels of this name ("" = all)
std::vector<Pending> g_pending;
std::vector<Stat> g_stats;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Launch one kernel through `fn`, counting it and, when profiling, timing it.
template <class F>
cudaError_t timed(const char* name, double algo_bytes, cudaStream_t st, F&& fn)
{
    if (g_launch_sink) {  // recorded into a graph: counted when the graph runs
        ++*g_launch_sink;
        return fn();
    }
    cudaEvent_t a = nullptr, b = nullptr;
    bool prof;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        prof = g_prof_on && (g_prof_only.empty() || g_prof_only == name);
        if (prof) {
            a = take_event();
            b = take_event();
        }
    }
    if (prof && a && b) cudaEventRecord(a, st);
    cudaError_t e = fn();
    g_launches.fetch_add(1);
    if (prof && a && b) {
        cudaEventRecord(b, st);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_pending.push_back({name, algo_bytes, a, b});
    }
    return e;
}

}  // namespace

namespace qai {
namespace host {

// ---- shapes -----------------------------------------------------------------
constexpr int kMaxX = 16383, kMaxYZ = 4096, kMax1D = 32768;

qai_status make_shape(int rank, const int64_t* dims, Shape* s)
{
    if (!dims) return fail(QAI_ERR_INVALID_ARG, "dims is NULL");
    if (rank < 1 || rank > 3) return fail(QAI_ERR_SHAPE, "rank %d outside 1..3", rank);
    int64_t kept[3];
    int r = 0;
    int64_t N = 1;
    for (int a = 0; a < rank; ++a) {
        if (dims[a] < 1) return fail(QAI_ERR_SHAPE, "dims[%d] = %lld < 1", a, (long long)dims[a]);
        if (dims[a] > (1LL << 31)) return fail(QAI_ERR_SHAPE, "dims[%d] too large", a);
        N *= dims[a];
        if (N >= (1LL << 31)) return fail(QAI_ERR_SHAPE, "N >= 2^31 points");
        if (dims[a] > 1) kept[r++] = dims[a];
    }
    if (r == 0) { kept[0] = 1; r = 1; }
    s->rank = r;
    s->N = N;
    s->nz = r == 3 ? (int)kept[0] : 1;
    s->ny = r >= 2 ? (int)kept[r - 2] : 1;
    s->nx = (int)kept[r - 1];
    if (r == 1 && s->nx > kMax1D)
        return fail(QAI_ERR_SHAPE, "rank-1 length %d > %d", s->nx, kMax1D);
    if (r >= 2 && s->nx > kMaxX)
        return fail(QAI_ERR_SHAPE, "x extent %d > %d", s->nx, kMaxX);
    if (r >= 2 && (s->ny > kMaxYZ || s->nz > kMaxYZ))
        return fail(QAI_ERR_SHAPE, "y or z extent > %d", kMaxYZ);
    return QAI_OK;
}

// ---- workspace layout -----------------------------------------------------------
size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

cudaError_t timed_call(const char* name, double algo_bytes, cudaStream_t st, const std::function<cudaError_t()>& fn)
{
    return timed(name, algo_bytes, st, fn);
}

Layout layout_for(const Shape& s, uint32_t flags)
{
    Layout l{};
    const size_t N = (size_t)s.N;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    l.eqm = take(N);
    l.dist1 = take(N * 4);
    l.s = take(N);
    l.xw = s.rank >= 2 ? take(N * 2) : 0;
    l.yw = s.rank >= 3 ? take(N * 4) : 0;
    l.idx = (flags & QAI_WS_INDEX) && s.rank >= 2 ? take(N * 4) : 0;
    // a uint16 count per column of the last column pass (z: ny * nx, y: nx)
    l.cflag = s.rank == 3 ? take((size_t)s.ny * s.nx * 2) : s.rank == 2 ? take((size_t)s.nx * 2) : 0;
    if (s.rank >= 2) {
        const size_t rows = (size_t)s.nz * s.ny;
        l.wpr = (s.nx + 15) / 16;
        l.bwpr = (s.nx + 31) / 32;
        l.codes = take(rows * l.wpr * 4);
        l.nexy = take(rows * l.wpr * 4);
        l.nez = s.rank == 3 ? take(rows * l.wpr * 4) : 0;
        l.spk = take(rows * l.wpr * 4);
        l.b2bits = take(rows * l.bwpr * 4);
        // the query lists: past them the dense second EDT takes over, which
        // in 3-D costs three passes over the field and the byte maps of the
        // separable passes -- about what the route spends on 3 % of the
        // points as queries; in 2-D its passes are cheap next to the route
        l.qcap = (int)(s.rank == 3 ? N / 32 + 1024 : N / 128 + 1024);
        l.scap = (int)(N / 256 + 1024);
        l.fcap = std::min(l.qcap, 1 << 16);
        l.b2cap = (int)(N / 32 + 4096);  // B2 sites up to ~3 % of the points
        l.ctr = take(qai::kCtrWords * 4);
        l.qlist = take((size_t)l.qcap * sizeof(qai::Query));
        l.slist = take((size_t)l.scap * 4);
        l.mlist = take((size_t)l.qcap * sizeof(qai::Query));
        l.flist = take((size_t)l.fcap * sizeof(qai::Query));
        l.fmin = take((size_t)l.fcap * 4);
        l.b2list = take((size_t)l.b2cap * 8);
    }
    l.total = off;
    return l;
}

bool plain_args(const int32_t* d_q, float* d_out, const Shape& sh, const qai::MethodArgs& m, char* ws,
                const Layout& lay, int* ctr, PlainArgs* pa)
{
    *pa = PlainArgs{};
    uint8_t* eqm = reinterpret_cast<uint8_t*>(ws + lay.eqm);
    int32_t* dist1 = reinterpret_cast<int32_t*>(ws + lay.dist1);
    int8_t* s = reinterpret_cast<int8_t*>(ws + lay.s);
    uint16_t* xw = reinterpret_cast<uint16_t*>(ws + lay.xw);
    uint32_t* yw = sh.rank >= 3 ? reinterpret_cast<uint32_t*>(ws + lay.yw) : nullptr;
    uint16_t* cflag = reinterpret_cast<uint16_t*>(ws + lay.cflag);
    qai::Query* qlist = reinterpret_cast<qai::Query*>(ws + lay.qlist);
    const int* local_fail = ctr + qai::kCtrLocalFail;
    const int* dense = ctr + qai::kCtrDense;
    const int64_t gx = (int64_t)(sh.nx - 1) * (sh.nx - 1);
    const int64_t gxy = gx + (int64_t)(sh.ny - 1) * (sh.ny - 1);
    auto al = [](const void* p, int b) { return (reinterpret_cast<uintptr_t>(p) % b) == 0; };

    qai::LocalArgs& la = pa->la;
    la.rank = sh.rank; la.nz = sh.nz; la.ny = sh.ny; la.nx = sh.nx; la.wpr = lay.wpr;
    la.q = d_q; la.out = d_out; la.ctr = ctr; la.dist1 = dist1;
    la.codes = reinterpret_cast<uint32_t*>(ws + lay.codes);
    la.nexy = reinterpret_cast<uint32_t*>(ws + lay.nexy);
    la.nez = sh.rank == 3 ? reinterpret_cast<uint32_t*>(ws + lay.nez) : nullptr;
    la.spk = reinterpret_cast<uint32_t*>(ws + lay.spk);
    la.qlist = qlist; la.qcap = lay.qcap;
    la.slist = reinterpret_cast<int32_t*>(ws + lay.slist); la.scap = lay.scap;
    la.eqm = eqm; la.s = s; la.m = m;
    la.vec = (sh.nx % 4 == 0) && al(d_q, 16) && al(d_out, 16);

    qai::RowArgs& r1 = pa->r1;
    r1.rank = sh.rank; r1.nz = sh.nz; r1.ny = sh.ny; r1.nx = sh.nx;
    r1.q = d_q; r1.eqm = eqm; r1.m = m;
    r1.out_pre = d_out; r1.route_ctr = ctr; r1.gate = local_fail;
    r1.xw = xw;
    qai::prepare_rowpass(r1);

    auto y_args = [&](const void* in) {
        qai::ColArgs c{};
        c.in = in; c.L = sh.ny; c.C = sh.nx; c.P = sh.nz;
        c.row_stride = sh.nx; c.plane_stride = (int64_t)sh.ny * sh.nx; c.m = m;
        return c;
    };
    auto z_args = [&](const void* in) {
        qai::ColArgs c{};
        c.in = in; c.L = sh.nz; c.C = sh.ny * sh.nx; c.P = 1;
        c.row_stride = (int64_t)sh.ny * sh.nx; c.plane_stride = 0; c.m = m;
        return c;
    };
    auto route_args = [&](qai::ColArgs& c) {
        c.route_ctr = ctr; c.qlist = qlist; c.qcap = lay.qcap;
        c.slist = reinterpret_cast<int32_t*>(ws + lay.slist); c.scap = lay.scap;
        c.gate = local_fail;
    };
    auto fuse_e = [&](qai::ColArgs& c) {
        c.out = d_out; c.q = d_q; c.dist1_in = dist1; c.s_in = s;
        c.col_count_in = nullptr;  // the local first EDT: B1 from the mask byte
        c.b1_eqm = eqm;
        c.route_ctr = ctr;
        c.gate = dense;
    };
    auto prep = [&](qai::ColArgs& c, int in_bytes, bool first_last, qai::ColConfig* cfg, int64_t max_g) {
        if (!qai::choose_colpass(c.L, in_bytes, cfg, first_last)) return false;
        qai::prepare_colpass(c, in_bytes, *cfg, max_g);
        return true;
    };
    if (sh.rank == 2) {
        pa->c1[0] = y_args(xw);
        pa->c1[0].dist1 = dist1; pa->c1[0].s_out = s; pa->c1[0].col_count_out = cflag;
        route_args(pa->c1[0]);
        pa->c2[0] = y_args(xw);
        fuse_e(pa->c2[0]);
        if (!prep(pa->c1[0], 2, true, &pa->cfg1[0], gx) || !prep(pa->c2[0], 2, false, &pa->cfg2[0], gx)) return false;
    } else {
        pa->c1[0] = y_args(xw);
        pa->c1[0].out_w = yw; pa->c1[0].gate = local_fail;
        pa->c1[1] = z_args(yw);
        pa->c1[1].dist1 = dist1; pa->c1[1].s_out = s; pa->c1[1].col_count_out = cflag;
        route_args(pa->c1[1]);
        pa->c2[0] = y_args(xw);
        pa->c2[0].out_w = yw; pa->c2[0].gate = dense;
        pa->c2[1] = z_args(yw);
        fuse_e(pa->c2[1]);
        if (!prep(pa->c1[0], 2, false, &pa->cfg1[0], gx) || !prep(pa->c1[1], 4, true, &pa->cfg1[1], gxy) ||
            !prep(pa->c2[0], 2, false, &pa->cfg2[0], gx) || !prep(pa->c2[1], 4, false, &pa->cfg2[1], gxy))
            return false;
    }

    qai::RouteArgs& ra = pa->ra;
    ra.rank = sh.rank; ra.nz = sh.nz; ra.ny = sh.ny; ra.nx = sh.nx;
    ra.wpr = lay.wpr; ra.bwpr = lay.bwpr;
    ra.q = d_q; ra.spk = la.spk; ra.nexy = la.nexy; ra.nez = la.nez; ra.out = d_out; ra.ctr = ctr;
    ra.slist = reinterpret_cast<const int32_t*>(ws + lay.slist); ra.scap = lay.scap;
    ra.b2bits = reinterpret_cast<uint32_t*>(ws + lay.b2bits);
    ra.qlist = qlist; ra.qcap = lay.qcap;
    ra.mlist = reinterpret_cast<qai::Query*>(ws + lay.mlist);
    ra.flist = reinterpret_cast<qai::Query*>(ws + lay.flist); ra.fcap = lay.fcap;
    ra.fmin = reinterpret_cast<int32_t*>(ws + lay.fmin);
    ra.b2list = reinterpret_cast<int32_t*>(ws + lay.b2list); ra.b2cap = lay.b2cap;
    ra.shell = 1;
    ra.d2rec = nullptr;
    ra.brute_budget = 1LL << 28;
    ra.m = m;

    qai::RowArgs& r2 = pa->r2;
    r2.rank = sh.rank; r2.nz = sh.nz; r2.ny = sh.ny; r2.nx = sh.nx;
    r2.q = d_q; r2.eqm = eqm; r2.s_in = s; r2.m = m;
    r2.xw = xw;
    r2.gate = dense;
    qai::prepare_rowpass(r2);
    return true;
}

qai_status check_params(const qai_params* p)
{
    if (!std::isfinite(p->eta) || p->eta < 0) return fail(QAI_ERR_INVALID_ARG, "eta must be finite and >= 0");
    if (!std::isfinite(p->idw_power) || p->idw_power <= 0)
        return fail(QAI_ERR_INVALID_ARG, "idw_power must be finite and > 0");
    if (p->grad_threshold < 1) return fail(QAI_ERR_INVALID_ARG, "grad_threshold must be >= 1");
    if (p->sign_rule != 0 && p->sign_rule != 1) return fail(QAI_ERR_INVALID_ARG, "sign_rule must be 0 or 1");
    if (p->b2_rule != 0 && p->b2_rule != 1) return fail(QAI_ERR_INVALID_ARG, "b2_rule must be 0 or 1");
    const uint32_t known = QAI_FLAG_OUTPUT_C | QAI_FLAG_EDT2_DENSE | QAI_FLAG_EDT2_HANDOVER | QAI_FLAG_EDT2_LIST |
                           QAI_FLAG_EDT1_SEPARABLE;
    if (p->flags & ~known) return fail(QAI_ERR_INVALID_ARG, "unknown bits in flags");
    const uint32_t e2 = p->flags & (QAI_FLAG_EDT2_DENSE | QAI_FLAG_EDT2_HANDOVER | QAI_FLAG_EDT2_LIST);
    if (e2 & (e2 - 1)) return fail(QAI_ERR_INVALID_ARG, "more than one QAI_FLAG_EDT2_* bit in flags");
    return QAI_OK;
}

qai::MethodArgs method_args(const qai_params* p, double eb)
{
    qai::MethodArgs m;
    m.two_eb = (float)(2.0 * eb);
    m.eta_eb = (float)(p->eta * eb);
    m.idw_power = (float)p->idw_power;
    m.idw_is_one = p->idw_power == 1.0;
    m.grad_threshold = p->grad_threshold;
    m.sign_rule = p->sign_rule;
    m.b2_rule = p->b2_rule;
    m.output_c = (p->flags & QAI_FLAG_OUTPUT_C) ? 1 : 0;
    m.flags = p->flags;
    return m;
}

qai_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(QAI_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace host
}  // namespace qai

namespace {
using namespace qai::host;

// Adjoint mode of the pipeline (rank 2 and 3): the last column pass sums the
// terms of dL/deta and dL/dp against grad_out instead of writing D''.
struct GradSink {
    const float* grad_out;
    double* partials;  // 2 doubles per CTA of the last pass
    int nblocks;       // set by run_pipeline
};

// Route of the second EDT for plain calls, from the route selection bits of
// qai_params.flags (testing and measurement only; all routes give the same
// bits): Off = the dense second EDT alone, Dense = the route's kernels run
// but hand every field to the dense second EDT, Brute = no shell search
// (every query goes to the brute-force search), Auto = the default.
enum class Route { Auto, Off, Dense, Brute };
Route signed_route(uint32_t flags)
{
    if (flags & QAI_FLAG_EDT2_DENSE) return Route::Off;
    if (flags & QAI_FLAG_EDT2_HANDOVER) return Route::Dense;
    if (flags & QAI_FLAG_EDT2_LIST) return Route::Brute;
    return Route::Auto;
}

// First EDT of plain calls with the signed-point route: the local search with
// the separable passes behind it (default), or the separable passes alone
// (QAI_FLAG_EDT1_SEPARABLE). Both give the same bits.
bool local_first_edt(uint32_t flags) { return !(flags & QAI_FLAG_EDT1_SEPARABLE); }

// CTAs of the last EDT2 pass (the sums it leaves in the partials array).
int final_pass_blocks(const Shape& sh)
{
    if (sh.rank == 1) return 0;
    const int L = sh.rank == 2 ? sh.ny : sh.nz, in_bytes = sh.rank == 2 ? 2 : 4;
    qai::ColConfig cfg;
    if (!qai::choose_colpass(L, in_bytes, &cfg)) return -1;
    qai::ColArgs c{};
    c.C = sh.rank == 2 ? sh.nx : sh.ny * sh.nx;
    c.P = sh.rank == 2 ? sh.nz : 1;
    return qai::colpass_blocks(c, cfg.W);
}

// The host-memory pipeline of qai_mitigate_host (see there): step A runs in
// z-slabs as their planes of q arrive, and each slab of D'' goes back while
// later slabs arrive.
constexpr int kMaxSlabs = 16;
struct HostPipe {
    const int32_t* h_q;
    float* h_out;          // host buffer, as the caller passed it
    float* h_out_dev;      // its device (mapped) address
    int nslab;
    int zb[kMaxSlabs + 1]; // slab k: planes zb[k] .. zb[k + 1] - 1
    cudaStream_t sin, sout;
    cudaEvent_t ev_in[kMaxSlabs], ev_a[kMaxSlabs], ev_out;
};

// The launch sequence of Algorithm 4 on a validated shape.
// d2rec (plain calls with the signed-point route only): Dist2 is recorded
// there, by point, wherever S != 0 off B1 (the adjoint's forward).
// saved (plain calls with the signed-point route only): the adjoint's saved
// state is written there (S everywhere; Dist1 and Dist2 where S != 0 off B1,
// 0 elsewhere); Dist2 is recorded straight into it.
qai_status run_pipeline(const int32_t* d_q, float* d_out, const Shape& sh, const qai::MethodArgs& m,
                        char* ws, const Layout& lay, cudaStream_t st, const qai_debug_out* dbg,
                        GradSink* grad = nullptr, int32_t* d2rec = nullptr, const qai_debug_out* saved = nullptr,
                        const HostPipe* hp = nullptr)
{
    if (saved) d2rec = saved->dist2;
    const double N = (double)sh.N;
    uint8_t* eqm = reinterpret_cast<uint8_t*>(ws + lay.eqm);
    int32_t* dist1 = reinterpret_cast<int32_t*>(ws + lay.dist1);
    int8_t* s = reinterpret_cast<int8_t*>(ws + lay.s);
    uint16_t* xw = sh.rank >= 2 ? reinterpret_cast<uint16_t*>(ws + lay.xw) : nullptr;
    uint32_t* yw = sh.rank >= 3 ? reinterpret_cast<uint32_t*>(ws + lay.yw) : nullptr;
    int32_t* idx_tmp = lay.idx ? reinterpret_cast<int32_t*>(ws + lay.idx) : nullptr;
    qai_debug_out none{};
    const qai_debug_out& d = dbg ? *dbg : none;
    const bool debug = d.b1 || d.sb || d.dist1 || d.idx1 || d.s || d.b2 || d.dist2;
    const int64_t gx = (int64_t)(sh.nx - 1) * (sh.nx - 1);           // max g after the x pass
    const int64_t gxy = gx + (int64_t)(sh.ny - 1) * (sh.ny - 1);     // after the y pass
    cudaError_t e;
    // The signed-point route: plain calls on rank 2 and 3 fields (the debug
    // maps and the adjoint need the dense second EDT everywhere).
    const Route route = signed_route(m.flags);
    const bool signed_route_on = !debug && !grad && sh.rank >= 2 && route != Route::Off;
    int* ctr = signed_route_on ? reinterpret_cast<int*>(ws + lay.ctr) : nullptr;
    const bool local = ctr && local_first_edt(m.flags);
    const int* local_fail = local ? ctr + qai::kCtrLocalFail : nullptr;  // gate of the separable first EDT
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ctr) {
        if ((e = cudaMemsetAsync(ctr, 0, qai::kCtrWords * sizeof(int), st)) != cudaSuccess)
            return cuda_fail(e, "route counters");
    }
    qai::LocalArgs la{};
    if (ctr) {
        la.rank = sh.rank; la.nz = sh.nz; la.ny = sh.ny; la.nx = sh.nx; la.wpr = lay.wpr;
        la.q = d_q; la.out = d_out; la.ctr = ctr; la.dist1 = dist1;
        la.codes = reinterpret_cast<uint32_t*>(ws + lay.codes);
        la.nexy = reinterpret_cast<uint32_t*>(ws + lay.nexy);
        la.nez = sh.rank == 3 ? reinterpret_cast<uint32_t*>(ws + lay.nez) : nullptr;
        la.spk = reinterpret_cast<uint32_t*>(ws + lay.spk);
        la.qlist = reinterpret_cast<qai::Query*>(ws + lay.qlist); la.qcap = lay.qcap;
        la.slist = reinterpret_cast<int32_t*>(ws + lay.slist); la.scap = lay.scap;
        la.eqm = eqm; la.s = s;
        la.m = m;
        auto al = [](const void* p, int b) { return (reinterpret_cast<uintptr_t>(p) % b) == 0; };
        la.vec = (sh.nx % 4 == 0) && al(d_q, 16) && al(d_out, 16);
    }
    if (ctr && hp) {
        // Step A slab by slab as q arrives, each slab of D'' back to the host
        // as soon as it is written; then the exact pass behind the slabs.
        // Step A at a plane needs the plane after it, so the launch after
        // copy k covers the planes from the last of copy k - 1 to the one
        // before the last of copy k (the last launch to the end).
        const size_t plane = (size_t)sh.ny * sh.nx;
        for (int k = 0; k < hp->nslab; ++k) {
            cudaStreamWaitEvent(st, hp->ev_in[k], 0);
            const int zb = k == 0 ? 0 : hp->zb[k] - 1;
            const int zn = (k + 1 == hp->nslab ? sh.nz : hp->zb[k + 1] - 1) - zb;
            e = timed("detect", (double)zn * plane * 8.75, st,
                      [&] { return qai::launch_local_detect_slab(la, zb, zn, st); });
            if (e != cudaSuccess) return cuda_fail(e, "step A (slab)");
            if ((e = cudaEventRecord(hp->ev_a[k], st)) != cudaSuccess) return cuda_fail(e, "event");
            if ((e = cudaStreamWaitEvent(hp->sout, hp->ev_a[k], 0)) != cudaSuccess) return cuda_fail(e, "event");
            e = cudaMemcpyAsync(hp->h_out + (size_t)zb * plane, d_out + (size_t)zb * plane,
                                (size_t)zn * plane * sizeof(float), cudaMemcpyDeviceToHost, hp->sout);
            if (e != cudaSuccess) return cuda_fail(e, "copy D'' slab to host");
        }
        if ((e = cudaEventRecord(hp->ev_out, hp->sout)) != cudaSuccess) return cuda_fail(e, "event");
        e = timed("detect", 0.0, st, [&] { return qai::launch_local_detect_exact(la, st); });
        if (e != cudaSuccess) return cuda_fail(e, "step A (exact pass)");
    } else if (ctr) {
        // Step A with the output where Dist2 does not matter and the packed
        // maps of the route (B1 with S_B, equal neighbours)
        e = timed("detect", N * (sh.rank == 3 ? 8.75 : 8.5), st, [&] { return qai::launch_local_detect(la, st); });
        if (e != cudaSuccess) return cuda_fail(e, "step A");
        if (m.sign_rule == 0) count_launch();  // the exact pass behind the fast one
    }
    if (local) {
        // Steps B and C by the bounded nearest-site search; the separable
        // passes below run only if some point has no B1 point within reach.
        e = timed("near", N * 0.5, st, [&] { return qai::launch_local_near(la, st); });
        if (e != cudaSuccess) return cuda_fail(e, "nearest-site search");
    }

    // Step A + EDT-x of B1 (rank 1: the whole first EDT).
    qai::RowArgs r1{};
    r1.rank = sh.rank; r1.nz = sh.nz; r1.ny = sh.ny; r1.nx = sh.nx;
    r1.q = d_q; r1.eqm = eqm; r1.m = m;
    r1.dbg_b1 = d.b1; r1.dbg_sb = d.sb;
    if (ctr) { r1.out_pre = d_out; r1.route_ctr = ctr; r1.gate = local_fail; }
    const bool final1 = sh.rank == 1;
    if (final1) { r1.dist1 = dist1; r1.s_out = s; r1.dbg_idx = d.idx1; }
    else { r1.xw = xw; r1.dbg_idx = d.idx1 ? (sh.rank == 3 ? d.idx1 : idx_tmp) : nullptr; }
    e = timed(final1 ? "rowpass1_final" : "rowpass1", N * (final1 ? 10.0 : 7.0), st,
              [&] { return qai::launch_rowpass(1, final1, r1, debug, st); });
    if (e != cudaSuccess) return cuda_fail(e, "row pass 1");

    // EDT1 along y (and z): Dist1 and the propagated sign S.
    auto colpass = [&](int phase, int in_bytes, bool fin, qai::ColArgs& c, const char* name,
                       double bytes_per_pt) -> qai_status {
        const int64_t max_g = in_bytes == 2 ? gx : gxy;
        qai::ColConfig cfg;
        if (!qai::choose_colpass(c.L, in_bytes, &cfg, phase == 1 && fin))
            return fail(QAI_ERR_SHAPE, "line length %d does not fit shared memory", c.L);
        cudaError_t err = timed(name, N * bytes_per_pt, st,
                                [&] { return qai::launch_colpass(phase, in_bytes, fin, c, cfg, debug, max_g, st); });
        if (err != cudaSuccess) return cuda_fail(err, name);
        return QAI_OK;
    };
    auto y_args = [&](const void* in) {
        qai::ColArgs c{};
        c.in = in; c.L = sh.ny; c.C = sh.nx; c.P = sh.nz;
        c.row_stride = sh.nx; c.plane_stride = (int64_t)sh.ny * sh.nx; c.m = m;
        return c;
    };
    auto z_args = [&](const void* in) {
        qai::ColArgs c{};
        c.in = in; c.L = sh.nz; c.C = sh.ny * sh.nx; c.P = 1;
        c.row_stride = (int64_t)sh.ny * sh.nx; c.plane_stride = 0; c.m = m;
        return c;
    };
    qai_status st_;
    uint16_t* cflag = sh.rank >= 2 ? reinterpret_cast<uint16_t*>(ws + lay.cflag) : nullptr;
    qai::Query* qlist = ctr ? reinterpret_cast<qai::Query*>(ws + lay.qlist) : nullptr;
    auto route_args = [&](qai::ColArgs& c) {
        if (!ctr) return;
        c.route_ctr = ctr; c.qlist = qlist; c.qcap = lay.qcap;
        c.slist = reinterpret_cast<int32_t*>(ws + lay.slist); c.scap = lay.scap;
        c.gate = local_fail;
    };
    if (sh.rank == 2) {
        qai::ColArgs c = y_args(xw);
        c.dist1 = dist1; c.s_out = s; c.col_count_out = cflag;
        route_args(c);
        if (d.idx1) { c.dbg_idx_in = idx_tmp; c.dbg_idx_out = d.idx1; }
        if ((st_ = colpass(1, 2, true, c, "colpass1_y_final", 2 + 4 + 1)) != QAI_OK) return st_;
    } else if (sh.rank == 3) {
        qai::ColArgs c = y_args(xw);
        c.out_w = yw;
        c.gate = local_fail;
        if (d.idx1) { c.dbg_idx_in = d.idx1; c.dbg_idx_out = idx_tmp; }
        if ((st_ = colpass(1, 2, false, c, "colpass1_y", 2 + 4)) != QAI_OK) return st_;
        qai::ColArgs cz = z_args(yw);
        cz.dist1 = dist1; cz.s_out = s; cz.col_count_out = cflag;
        route_args(cz);
        if (d.idx1) { cz.dbg_idx_in = idx_tmp; cz.dbg_idx_out = d.idx1; }
        if ((st_ = colpass(1, 4, true, cz, "colpass1_z_final", 4 + 4 + 1)) != QAI_OK) return st_;
    }
    if (ctr) {  // the packed S of the route, from the separable first EDT's S map when it ran
        e = timed("pack_s", N * 1.25, st, [&] { return qai::launch_local_pack_s(la, local, st); });
        if (e != cudaSuccess) return cuda_fail(e, "packed S");
    }
    if (d.dist1 && (e = cudaMemcpyAsync(d.dist1, dist1, (size_t)sh.N * 4, cudaMemcpyDeviceToDevice, st)))
        return cuda_fail(e, "copy dist1");
    if (d.s && (e = cudaMemcpyAsync(d.s, s, (size_t)sh.N, cudaMemcpyDeviceToDevice, st)))
        return cuda_fail(e, "copy s");

    // Signed-point route: exact Dist2 and step E at the queries; the dense
    // second EDT below runs only if this route hands the field over.
    if (ctr) {
        qai::RouteArgs ra{};
        ra.rank = sh.rank; ra.nz = sh.nz; ra.ny = sh.ny; ra.nx = sh.nx;
        ra.wpr = lay.wpr; ra.bwpr = lay.bwpr;
        ra.q = d_q; ra.spk = la.spk; ra.nexy = la.nexy; ra.nez = la.nez; ra.out = d_out; ra.ctr = ctr;
        ra.slist = reinterpret_cast<const int32_t*>(ws + lay.slist); ra.scap = lay.scap;
        ra.b2bits = reinterpret_cast<uint32_t*>(ws + lay.b2bits);
        ra.qlist = qlist; ra.qcap = lay.qcap;
        ra.mlist = reinterpret_cast<qai::Query*>(ws + lay.mlist);
        ra.flist = reinterpret_cast<qai::Query*>(ws + lay.flist); ra.fcap = lay.fcap;
        ra.fmin = reinterpret_cast<int32_t*>(ws + lay.fmin);
        ra.b2list = reinterpret_cast<int32_t*>(ws + lay.b2list); ra.b2cap = lay.b2cap;
        ra.shell = route == Route::Brute ? 0 : 1;
        ra.d2rec = d2rec;
        ra.brute_budget = 1LL << 28;
        ra.m = m;
        if (route == Route::Dense) ra.qcap = -1;  // every count is over it: hand over at once
        // the sparse route: B2 sites from the signed set, every query against them
        e = timed("b2sparse", 0.0, st, [&] { return qai::launch_route_sparse_sites(ra, st); });
        if (e != cudaSuccess) return cuda_fail(e, "B2 sites of the signed set");
        e = timed("brute_sparse", 0.0, st, [&] { return qai::launch_route_brute(ra, 2 * sms, true, st); });
        if (e != cudaSuccess) return cuda_fail(e, "search over the B2 sites");
        // the bitmap route, when the sparse one could not run
        e = timed("b2map", N * (sh.rank == 3 ? 1.125 : 0.875), st, [&] { return qai::launch_route_b2map(ra, st); });
        if (e != cudaSuccess) return cuda_fail(e, "B2 bitmap");
        e = timed("signed_query", 0.0, st, [&] { return qai::launch_route_query(ra, 4 * sms, st); });
        if (e != cudaSuccess) return cuda_fail(e, "signed-point shell search");
        e = timed("signed_query_mid", 0.0, st, [&] { return qai::launch_route_query_mid(ra, 4 * sms, st); });
        if (e != cudaSuccess) return cuda_fail(e, "signed-point shell search, second phase");
        e = timed("b2list", 0.0, st, [&] { return qai::launch_route_b2list(ra, st); });
        if (e != cudaSuccess) return cuda_fail(e, "B2 site list");
        e = timed("signed_brute", 0.0, st, [&] { return qai::launch_route_brute(ra, 2 * sms, false, st); });
        if (e != cudaSuccess) return cuda_fail(e, "brute-force search");
        // the byte maps of the separable passes, for the dense second EDT
        // when it takes over (the adjoint reads the packed maps)
        if (local) {
            e = timed("expand", 0.0, st, [&] { return qai::launch_local_expand(la, 1, st); });
            if (e != cudaSuccess) return cuda_fail(e, "byte maps");
        }
    }

    // B2 = GetBoundary(S) + EDT-x of B2 (rank 1: also step E).
    qai::RowArgs r2{};
    r2.rank = sh.rank; r2.nz = sh.nz; r2.ny = sh.ny; r2.nx = sh.nx;
    r2.q = d_q; r2.eqm = eqm; r2.s_in = s; r2.m = m;
    r2.dbg_b2 = d.b2;
    if (final1) { r2.dist1_in = dist1; r2.out = d_out; r2.dbg_dist2 = d.dist2; }
    else r2.xw = xw;
    r2.gate = ctr ? ctr + qai::kCtrDense : nullptr;
    e = timed(final1 ? "rowpass2_final" : "rowpass2", N * (final1 ? 14.0 : 4.0), st,
              [&] { return qai::launch_rowpass(2, final1, r2, debug, st); });
    if (e != cudaSuccess) return cuda_fail(e, "row pass 2");

    // EDT2 along y (and z), the last pass fused with step E.
    auto fuse_e = [&](qai::ColArgs& c) {
        c.out = d_out; c.q = d_q; c.dist1_in = dist1; c.s_in = s; c.dbg_dist2 = d.dist2;
        // the per-column counts exist only when the separable first EDT ran;
        // after the local one, B1 comes from the mask byte (Dist1 = 0 there
        // is not stored) -- the separable passes, when they ran, rewrote the
        // mask bytes on B1 without clearing any other bit pattern's meaning
        c.col_count_in = local ? nullptr : cflag;
        c.b1_eqm = local ? eqm : nullptr;
        c.d2rec = ctr ? d2rec : nullptr;
        c.route_ctr = ctr;
        c.gate = ctr ? ctr + qai::kCtrDense : nullptr;
    };
    // Adjoint mode: the last pass reads G, Dist1, S and the input words.
    auto last_grad = [&](qai::ColArgs& c, int in_bytes, const char* name) -> qai_status {
        c.dist1_in = dist1; c.s_in = s; c.grad_out = grad->grad_out; c.partials = grad->partials;
        c.col_count_in = cflag;
        qai::ColConfig cfg;
        if (!qai::choose_colpass(c.L, in_bytes, &cfg))
            return fail(QAI_ERR_SHAPE, "line length %d does not fit shared memory", c.L);
        grad->nblocks = qai::colpass_blocks(c, cfg.W);
        cudaError_t err = timed(name, N * (in_bytes + 4 + 1 + 4), st, [&] {
            return qai::launch_colpass_grad(in_bytes, c, cfg, in_bytes == 2 ? gx : gxy, st);
        });
        return err == cudaSuccess ? QAI_OK : cuda_fail(err, name);
    };
    if (sh.rank == 2) {
        qai::ColArgs c = y_args(xw);
        if (grad) return last_grad(c, 2, "colpass2_y_grad");
        fuse_e(c);
        if ((st_ = colpass(2, 2, true, c, "colpass2_y_final", 2 + 4 + 1 + 4 + 4)) != QAI_OK) return st_;
    } else if (sh.rank == 3) {
        qai::ColArgs c = y_args(xw);
        c.out_w = yw;
        c.gate = ctr ? ctr + qai::kCtrDense : nullptr;
        if ((st_ = colpass(2, 2, false, c, "colpass2_y", 2 + 4)) != QAI_OK) return st_;
        qai::ColArgs cz = z_args(yw);
        if (grad) return last_grad(cz, 4, "colpass2_z_grad");
        fuse_e(cz);
        if ((st_ = colpass(2, 4, true, cz, "colpass2_z_final", 4 + 4 + 1 + 4 + 4)) != QAI_OK) return st_;
    }
    if (saved && ctr) {
        e = timed("save", N * 9.5, st, [&] {
            return qai::launch_save_packed(la, saved->s, saved->dist1, saved->dist2, st);
        });
        if (e != cudaSuccess) return cuda_fail(e, "saved state");
    }
    if (hp) {
        // after the last slab's copy: what changed since, into the host buffer
        if ((e = cudaStreamWaitEvent(st, hp->ev_out, 0)) != cudaSuccess) return cuda_fail(e, "event");
        e = timed("host_fixup", 0.0, st, [&] { return qai::launch_host_fixup(la, hp->h_out_dev, st); });
        if (e != cudaSuccess) return cuda_fail(e, "host output fix-up");
    }
    return QAI_OK;
}

}  // namespace

namespace qai {
namespace host {

LaunchSink::LaunchSink(int* counter) : prev_(g_launch_sink) { g_launch_sink = counter; }
LaunchSink::~LaunchSink() { g_launch_sink = prev_; }

qai_status run_plain(const int32_t* d_q, float* d_out, const Shape& sh, const MethodArgs& m, char* ws,
                     const Layout& lay, cudaStream_t st)
{
    return run_pipeline(d_q, d_out, sh, m, ws, lay, st, nullptr);
}

}  // namespace host
}  // namespace qai

void qai::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

extern "C" {

void qai_default_params(qai_params* p)
{
    if (!p) return;
    p->eta = 0.9;
    p->idw_power = 1.0;
    p->grad_threshold = 2;
    p->sign_rule = 0;
    p->b2_rule = 0;
    p->flags = 0;
}

qai_status qai_workspace_size(int rank, const int64_t* dims, uint32_t flags, size_t* bytes)
{
    if (!bytes) return fail(QAI_ERR_INVALID_ARG, "bytes is NULL");
    Shape sh;
    qai_status s = make_shape(rank, dims, &sh);
    if (s != QAI_OK) return s;
    *bytes = layout_for(sh, flags).total;
    return QAI_OK;
}

}  // extern "C"

namespace {
// qai_mitigate with the adjoint's saved state written on the way (saved: the
// plain path with the signed-point route; see run_pipeline).
qai_status mitigate_impl(const int32_t* d_q, float* d_out, int rank, const int64_t* dims, double eb,
                         const qai_params* params, void* d_ws, size_t ws_bytes, cudaStream_t stream,
                         const qai_debug_out* dbg, const qai_debug_out* saved)
{
    if (!d_q || !d_out) return fail(QAI_ERR_INVALID_ARG, "d_q and d_out must be non-NULL");
    if (!(eb > 0.0) || !std::isfinite(eb)) return fail(QAI_ERR_INVALID_ARG, "eb must be finite and > 0");
    qai_params defaults;
    qai_default_params(&defaults);
    const qai_params* p = params ? params : &defaults;
    qai_status s = check_params(p);
    if (s != QAI_OK) return s;
    Shape sh;
    if ((s = make_shape(rank, dims, &sh)) != QAI_OK) return s;
    const uint32_t wflags = (dbg && dbg->idx1) ? QAI_WS_INDEX : 0u;
    const Layout lay = layout_for(sh, wflags);
    bool owned = false;
    if (d_ws) {
        if (ws_bytes < lay.total)
            return fail(QAI_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", ws_bytes, lay.total);
        if (reinterpret_cast<uintptr_t>(d_ws) & 255)
            return fail(QAI_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    } else {
        cudaError_t e = cudaMallocAsync(&d_ws, lay.total, stream);
        if (e != cudaSuccess) return fail(QAI_ERR_OOM, "cudaMallocAsync(%zu): %s", lay.total, cudaGetErrorString(e));
        owned = true;
    }
    s = run_pipeline(d_q, d_out, sh, method_args(p, eb), static_cast<char*>(d_ws), lay, stream, dbg, nullptr,
                     nullptr, saved);
    if (owned) cudaFreeAsync(d_ws, stream);
    return s;
}
}  // namespace

namespace {
// Internal streams and events of the host-memory pipeline, per device; one
// call enqueues at a time.
struct PipeRes {
    bool ready = false;
    cudaStream_t sin = nullptr, sout = nullptr;
    cudaEvent_t fork = nullptr, ev_in[kMaxSlabs] = {}, ev_a[kMaxSlabs] = {}, ev_out = nullptr;
};
std::mutex g_pipe_mu;
PipeRes g_pipe[64];

// The pipelined form needs the tiled step A (3-D rows of 16-byte multiples,
// aligned device buffers, the sign rule SUM), the route of plain calls, at
// least two slabs of planes, page-locked q and a page-locked, device-mapped
// output buffer.
bool host_pipeline_fits(const Shape& sh, const qai_params& p, const int32_t* h_q, const float* h_out,
                        const int32_t* d_q, const float* d_out)
{
    if (sh.rank != 3 || sh.nz < 16 || sh.nx % 4 != 0 || p.sign_rule != 0) return false;
    if (p.flags & (QAI_FLAG_EDT2_DENSE | QAI_FLAG_EDT1_SEPARABLE)) return false;
    if ((reinterpret_cast<uintptr_t>(d_q) | reinterpret_cast<uintptr_t>(d_out)) & 15) return false;
    cudaPointerAttributes aq{}, ao{};
    if (cudaPointerGetAttributes(&aq, h_q) != cudaSuccess || cudaPointerGetAttributes(&ao, h_out) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return aq.type == cudaMemoryTypeHost && ao.type == cudaMemoryTypeHost && ao.devicePointer != nullptr;
}

qai_status mitigate_host_pipelined(const int32_t* h_q, float* h_out, const Shape& sh, const qai_params* p, double eb,
                                   int32_t* d_q, float* d_out, char* ws, size_t ws_bytes, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return cuda_fail(e, "current device");
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    PipeRes& r = g_pipe[dev];
    if (!r.ready) {
        bool ok = cudaStreamCreateWithFlags(&r.sin, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&r.sout, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&r.ev_out, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ok && k < kMaxSlabs; ++k)
            ok = cudaEventCreateWithFlags(&r.ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&r.ev_a[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) return cuda_fail(cudaGetLastError(), "pipeline streams and events");
        r.ready = true;
    }
    cudaPointerAttributes ao{};
    if ((e = cudaPointerGetAttributes(&ao, h_out)) != cudaSuccess) return cuda_fail(e, "output buffer");
    HostPipe hp{};
    hp.h_q = h_q;
    hp.h_out = h_out;
    hp.h_out_dev = static_cast<float*>(ao.devicePointer);
    hp.nslab = std::min(kMaxSlabs, sh.nz / 8);
    for (int k = 0; k <= hp.nslab; ++k) hp.zb[k] = (int)((int64_t)sh.nz * k / hp.nslab);
    hp.sin = r.sin;
    hp.sout = r.sout;
    for (int k = 0; k < kMaxSlabs; ++k) {
        hp.ev_in[k] = r.ev_in[k];
        hp.ev_a[k] = r.ev_a[k];
    }
    hp.ev_out = r.ev_out;
    // both side streams start after the work already on `stream` (the last
    // call on this workspace may still read q and write D'')
    if ((e = cudaEventRecord(r.fork, st)) != cudaSuccess) return cuda_fail(e, "event");
    if ((e = cudaStreamWaitEvent(r.sin, r.fork, 0)) != cudaSuccess) return cuda_fail(e, "event");
    if ((e = cudaStreamWaitEvent(r.sout, r.fork, 0)) != cudaSuccess) return cuda_fail(e, "event");
    const size_t plane = (size_t)sh.ny * sh.nx;
    for (int k = 0; k < hp.nslab; ++k) {
        const size_t off = (size_t)hp.zb[k] * plane, n = (size_t)(hp.zb[k + 1] - hp.zb[k]) * plane;
        if ((e = cudaMemcpyAsync(d_q + off, h_q + off, n * 4, cudaMemcpyHostToDevice, r.sin)) != cudaSuccess)
            return cuda_fail(e, "copy q slab to device");
        if ((e = cudaEventRecord(r.ev_in[k], r.sin)) != cudaSuccess) return cuda_fail(e, "event");
    }
    const Layout lay = layout_for(sh, 0);
    if (ws_bytes < lay.total) return fail(QAI_ERR_INVALID_ARG, "workspace too small");
    return run_pipeline(d_q, d_out, sh, method_args(p, eb), ws, lay, st, nullptr, nullptr, nullptr, nullptr, &hp);
}
}  // namespace

extern "C" {

qai_status qai_mitigate(const int32_t* d_q, float* d_out, int rank, const int64_t* dims, double eb,
                        const qai_params* params, void* d_ws, size_t ws_bytes, cudaStream_t stream,
                        const qai_debug_out* dbg)
{
    g_last_error.clear();
    return mitigate_impl(d_q, d_out, rank, dims, eb, params, d_ws, ws_bytes, stream, dbg, nullptr);
}

qai_status qai_route_counts(const void* d_ws, int rank, const int64_t* dims, int32_t* counts,
                            cudaStream_t stream)
{
    g_last_error.clear();
    if (!d_ws || !counts) return fail(QAI_ERR_INVALID_ARG, "d_ws and counts must be non-NULL");
    Shape sh;
    qai_status s = make_shape(rank, dims, &sh);
    if (s != QAI_OK) return s;
    if (sh.rank < 2) return fail(QAI_ERR_SHAPE, "rank-1 fields have no signed-point route");
    const Layout lay = layout_for(sh, 0);
    int32_t c[qai::kCtrWords];
    cudaError_t e = cudaMemcpyAsync(c, static_cast<const char*>(d_ws) + lay.ctr, sizeof c,
                                    cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "read route counters");
    counts[0] = c[qai::kCtrQueries];
    counts[1] = c[qai::kCtrUnresolved];
    counts[2] = c[qai::kCtrB2];
    counts[3] = c[qai::kCtrDense] != 0;
    counts[4] = c[qai::kCtrSignedOver] ? -1 : c[c[qai::kCtrWide] ? qai::kCtrSignedExact : qai::kCtrSigned];
    counts[5] = c[qai::kCtrLocalFail] != 0;
    if (c[qai::kCtrTimeout])
        return fail(QAI_ERR_TIMEOUT, "a bounded device-side wait of that call ran out: its output is not valid");
    return QAI_OK;
}

qai_status qai_workspace_size_host(int rank, const int64_t* dims, size_t* bytes)
{
    if (!bytes) return fail(QAI_ERR_INVALID_ARG, "bytes is NULL");
    Shape sh;
    qai_status s = make_shape(rank, dims, &sh);
    if (s != QAI_OK) return s;
    *bytes = align256((size_t)sh.N * 4) * 2 + layout_for(sh, 0).total;
    return QAI_OK;
}

qai_status qai_mitigate_host(const int32_t* h_q, float* h_out, int rank, const int64_t* dims, double eb,
                             const qai_params* params, void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    g_last_error.clear();
    if (!h_q || !h_out || !d_ws) return fail(QAI_ERR_INVALID_ARG, "h_q, h_out and d_ws must be non-NULL");
    Shape sh;
    qai_status s = make_shape(rank, dims, &sh);
    if (s != QAI_OK) return s;
    const size_t fb = align256((size_t)sh.N * 4);
    size_t need;
    qai_workspace_size_host(rank, dims, &need);
    if (ws_bytes < need) return fail(QAI_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", ws_bytes, need);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return fail(QAI_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    char* base = static_cast<char*>(d_ws);
    int32_t* d_q = reinterpret_cast<int32_t*>(base);
    float* d_out = reinterpret_cast<float*>(base + fb);
    qai_params defaults;
    qai_default_params(&defaults);
    const qai_params* p = params ? params : &defaults;
    if ((s = check_params(p)) != QAI_OK) return s;
    if (!(eb > 0.0) || !std::isfinite(eb)) return fail(QAI_ERR_INVALID_ARG, "eb must be finite and > 0");
    cudaError_t e;
    if (host_pipeline_fits(sh, *p, h_q, h_out, d_q, d_out)) {
        // the pipelined form: q in slabs on one stream, step A per slab on
        // `stream` as they land, D'' slabs back on another as soon as step A
        // wrote them (the link carries both directions at once); the outputs
        // the later kernels change go straight into the mapped host buffer
        return mitigate_host_pipelined(h_q, h_out, sh, p, eb, d_q, d_out, base + 2 * fb, ws_bytes - 2 * fb, stream);
    }
    e = cudaMemcpyAsync(d_q, h_q, (size_t)sh.N * 4, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy q to device");
    s = qai_mitigate(d_q, d_out, rank, dims, eb, params, base + 2 * fb, ws_bytes - 2 * fb, stream, nullptr);
    if (s != QAI_OK) return s;
    e = cudaMemcpyAsync(h_out, d_out, (size_t)sh.N * 4, cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy D'' to host");
    return QAI_OK;
}

qai_status qai_saved_size(int rank, const int64_t* dims, size_t* bytes)
{
    if (!bytes) return fail(QAI_ERR_INVALID_ARG, "bytes is NULL");
    Shape sh;
    qai_status s = make_shape(rank, dims, &sh);
    if (s != QAI_OK) return s;
    *bytes = align256((size_t)sh.N * 4) * 2 + align256((size_t)sh.N);
    return QAI_OK;
}

// Saved state of the adjoint: Dist1 (int32), Dist2 (int32), S (int8).
static qai_debug_out saved_views(void* d_saved, int64_t N)
{
    char* b = static_cast<char*>(d_saved);
    qai_debug_out d{};
    d.dist1 = reinterpret_cast<int32_t*>(b);
    d.dist2 = reinterpret_cast<int32_t*>(b + align256((size_t)N * 4));
    d.s = reinterpret_cast<int8_t*>(b + 2 * align256((size_t)N * 4));
    return d;
}

qai_status qai_mitigate_save(const int32_t* d_q, float* d_out, int rank, const int64_t* dims, double eb,
                             const qai_params* params, void* d_saved, void* d_ws, size_t ws_bytes,
                             cudaStream_t stream)
{
    g_last_error.clear();
    if (!d_saved) return fail(QAI_ERR_INVALID_ARG, "d_saved must be non-NULL");
    if (reinterpret_cast<uintptr_t>(d_saved) & 255) return fail(QAI_ERR_INVALID_ARG, "d_saved must be 256-byte aligned");
    Shape sh;
    qai_status s = make_shape(rank, dims, &sh);
    if (s != QAI_OK) return s;
    const qai_debug_out d = saved_views(d_saved, sh.N);
    // rank 2 and 3: the plain path writes the saved state (Dist1 and Dist2
    // where S != 0 off B1, the only points whose terms are not zero); rank 1
    // (and the dense-only test route): the per-step maps of a debug call
    if (sh.rank >= 2 && signed_route(params ? params->flags : 0u) != Route::Off)
        return mitigate_impl(d_q, d_out, rank, dims, eb, params, d_ws, ws_bytes, stream, nullptr, &d);
    return mitigate_impl(d_q, d_out, rank, dims, eb, params, d_ws, ws_bytes, stream, &d, nullptr);
}

qai_status qai_dequantize(const int32_t* d_q, float* d_out, int64_t n, double eb, cudaStream_t stream)
{
    g_last_error.clear();
    if (!d_q || !d_out) return fail(QAI_ERR_INVALID_ARG, "d_q and d_out must be non-NULL");
    if (n < 0) return fail(QAI_ERR_INVALID_ARG, "n must be >= 0");
    if (!(eb > 0.0) || !std::isfinite(eb)) return fail(QAI_ERR_INVALID_ARG, "eb must be finite and > 0");
    if (n == 0) return QAI_OK;
    cudaError_t e = timed("dequantize", (double)n * 8, stream,
                          [&] { return qai::launch_dequantize(d_q, d_out, n, (float)(2.0 * eb), stream); });
    return e == cudaSuccess ? QAI_OK : cuda_fail(e, "dequantize");
}

qai_status qai_mitigate_add(const int32_t* d_q, const float* d_dprime, float* d_out, int rank, const int64_t* dims,
                            double eb, const qai_params* params, void* d_saved, void* d_ws, size_t ws_bytes,
                            cudaStream_t stream)
{
    g_last_error.clear();
    if (!d_dprime) return fail(QAI_ERR_INVALID_ARG, "d_dprime must be non-NULL");
    qai_params p;
    if (params) p = *params;
    else qai_default_params(&p);
    p.flags |= QAI_FLAG_OUTPUT_C;
    Shape sh;
    qai_status s = make_shape(rank, dims, &sh);
    if (s != QAI_OK) return s;
    s = d_saved ? qai_mitigate_save(d_q, d_out, rank, dims, eb, &p, d_saved, d_ws, ws_bytes, stream)
                : qai_mitigate(d_q, d_out, rank, dims, eb, &p, d_ws, ws_bytes, stream, nullptr);
    if (s != QAI_OK) return s;
    cudaError_t e = timed("add_dprime", (double)sh.N * 12, stream,
                          [&] { return qai::launch_add_dprime(d_dprime, d_out, sh.N, stream); });
    return e == cudaSuccess ? QAI_OK : cuda_fail(e, "D' + C");
}

}  // extern "C"

namespace {
// Partials of the adjoint: one pair per block of k_backward, or per CTA of
// the last column pass when that pass computes the sums.
size_t backward_partials_bytes(const Shape& sh, bool recompute)
{
    int64_t n = qai::kBackwardMaxBlocks;
    if (recompute) n = std::max<int64_t>(n, final_pass_blocks(sh));
    return align256(2 * sizeof(double) * (size_t)n);
}

// Recompute mode: the forward workspace plus room for D'' and Dist2.
size_t recompute_bytes(const Shape& sh)
{
    return layout_for(sh, 0).total + 2 * align256((size_t)sh.N * 4);
}
}  // namespace

extern "C" {

qai_status qai_workspace_size_backward(int rank, const int64_t* dims, int recompute, size_t* bytes)
{
    if (!bytes) return fail(QAI_ERR_INVALID_ARG, "bytes is NULL");
    Shape sh;
    qai_status s = make_shape(rank, dims, &sh);
    if (s != QAI_OK) return s;
    *bytes = backward_partials_bytes(sh, recompute != 0) + (recompute ? recompute_bytes(sh) : 0);
    return QAI_OK;
}

qai_status qai_mitigate_backward(const int32_t* d_q, const float* d_grad_out, float* d_grad_dprime,
                                 double* d_grad_params, int rank, const int64_t* dims, double eb,
                                 const qai_params* params, const void* d_saved, void* d_ws,
                                 size_t ws_bytes, cudaStream_t stream)
{
    g_last_error.clear();
    if (!d_q || !d_grad_out || !d_grad_params)
        return fail(QAI_ERR_INVALID_ARG, "d_q, d_grad_out and d_grad_params must be non-NULL");
    if (!(eb > 0.0) || !std::isfinite(eb)) return fail(QAI_ERR_INVALID_ARG, "eb must be finite and > 0");
    qai_params defaults;
    qai_default_params(&defaults);
    const qai_params* p = params ? params : &defaults;
    qai_status s = check_params(p);
    if (s != QAI_OK) return s;
    Shape sh;
    if ((s = make_shape(rank, dims, &sh)) != QAI_OK) return s;
    qai::BackArgs b{};
    b.N = sh.N;
    b.grad_out = d_grad_out;
    b.grad_dprime = d_grad_dprime;
    b.grad_params = d_grad_params;
    b.p = (float)p->idw_power;
    b.eta = p->eta;
    b.eb = eb;
    if (final_pass_blocks(sh) < 0) return fail(QAI_ERR_SHAPE, "line length does not fit shared memory");
    const size_t partials = backward_partials_bytes(sh, !d_saved);
    const size_t need = partials + (d_saved ? 0 : recompute_bytes(sh));
    if (!d_ws || ws_bytes < need)
        return fail(QAI_ERR_INVALID_ARG, "the adjoint needs a workspace of %zu bytes", need);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255) return fail(QAI_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    b.partials = static_cast<double*>(d_ws);
    cudaError_t e;
    if (d_saved) {
        const qai_debug_out v = saved_views(const_cast<void*>(d_saved), sh.N);
        b.dist1 = v.dist1;
        b.dist2 = v.dist2;
        b.s = v.s;
    } else if (sh.rank >= 2 && signed_route(p->flags) != Route::Off) {
        // recompute with the plain path: S everywhere, Dist1 and (recorded)
        // Dist2 wherever S != 0 off B1 -- the only points whose terms are not
        // zero; B1 points (Dist1 = 0) come from the mask bytes
        const Layout lay = layout_for(sh, 0);
        char* ws = static_cast<char*>(d_ws) + partials;
        float* scratch_out = reinterpret_cast<float*>(ws + lay.total);
        int32_t* d2rec = reinterpret_cast<int32_t*>(ws + lay.total + align256((size_t)sh.N * 4));
        s = run_pipeline(d_q, scratch_out, sh, method_args(p, eb), ws, lay, stream, nullptr, nullptr, d2rec);
        if (s != QAI_OK) return s;
        b.spk = reinterpret_cast<const uint32_t*>(ws + lay.spk);
        b.codes = reinterpret_cast<const uint32_t*>(ws + lay.codes);
        b.wpr = lay.wpr;
        b.nx = sh.nx;
        b.dist1 = reinterpret_cast<int32_t*>(ws + lay.dist1);
        b.dist2 = d2rec;
        if (d_grad_dprime &&
            (e = cudaMemcpyAsync(d_grad_dprime, d_grad_out, (size_t)sh.N * 4, cudaMemcpyDeviceToDevice, stream)))
            return cuda_fail(e, "copy dL/dD'");
        b.grad_dprime = nullptr;
    } else if (sh.rank >= 2) {
        // the dense-only route: recompute Dist1, S and the EDT2 words with
        // the dense pipeline; its last column pass sums the adjoint terms in
        // place of writing D''
        const Layout lay = layout_for(sh, 0);
        GradSink g{d_grad_out, b.partials, 0};
        s = run_pipeline(d_q, nullptr, sh, method_args(p, eb), static_cast<char*>(d_ws) + partials, lay,
                         stream, nullptr, &g);
        if (s != QAI_OK) return s;
        if (d_grad_dprime &&
            (e = cudaMemcpyAsync(d_grad_dprime, d_grad_out, (size_t)sh.N * 4, cudaMemcpyDeviceToDevice, stream)))
            return cuda_fail(e, "copy dL/dD'");
        e = timed("backward_sum", (double)g.nblocks * 16, stream, [&] {
            return qai::launch_partials_sum(b.partials, g.nblocks, eb, p->eta, d_grad_params, stream);
        });
        return e == cudaSuccess ? QAI_OK : cuda_fail(e, "backward sum");
    } else {
        // rank 1: recompute Dist1, S and Dist2 with the forward pipeline
        const Layout lay = layout_for(sh, 0);
        char* ws = static_cast<char*>(d_ws) + partials;
        int32_t* dist2 = reinterpret_cast<int32_t*>(ws + lay.total);
        float* scratch_out = reinterpret_cast<float*>(ws + lay.total + align256((size_t)sh.N * 4));
        qai_debug_out d{};
        d.dist2 = dist2;
        s = run_pipeline(d_q, scratch_out, sh, method_args(p, eb), ws, lay, stream, &d);
        if (s != QAI_OK) return s;
        b.dist1 = reinterpret_cast<int32_t*>(ws + lay.dist1);
        b.s = reinterpret_cast<int8_t*>(ws + lay.s);
        b.dist2 = dist2;
    }
    e = timed("backward", (double)sh.N * (4 + 1 + 4 + 4 + (d_grad_dprime ? 4 : 0)), stream,
              [&] { return qai::launch_backward(b, stream); });
    count_launch();  // the one-block combine
    if (e != cudaSuccess) return cuda_fail(e, "backward");
    return QAI_OK;
}

}  // extern "C"

namespace {
constexpr int kQualStatBlocks = 1024;

// The window grid of qai_quality on a validated shape (readings in qai.h).
qai::QualArgs quality_args(const Shape& sh, int window, int stride)
{
    qai::QualArgs a{};
    a.nz = sh.nz; a.ny = sh.ny; a.nx = sh.nx;
    auto axis = [&](int n, int* m, int* s, int* nw) {
        *m = n > 1 ? std::min(window, n) : 1;
        *s = n > 1 ? stride : 1;
        *nw = (n - *m) / *s + 1;
    };
    axis(sh.nz, &a.mz, &a.sz, &a.nwz);
    axis(sh.ny, &a.my, &a.sy, &a.nwy);
    axis(sh.nx, &a.mx, &a.sx, &a.nwx);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    qai::plan_quality(a, sms);
    return a;
}

size_t quality_stat_bytes() { return align256(3 * sizeof(double) * kQualStatBlocks); }

qai_status check_window(int window, int stride)
{
    if (window < 1 || window > 11) return fail(QAI_ERR_INVALID_ARG, "window %d outside 1..11", window);
    if (stride < 1 || stride > 4) return fail(QAI_ERR_INVALID_ARG, "stride %d outside 1..4", stride);
    return QAI_OK;
}
}  // namespace

extern "C" {

qai_status qai_workspace_size_quality(int rank, const int64_t* dims, int window, int stride, size_t* bytes)
{
    if (!bytes) return fail(QAI_ERR_INVALID_ARG, "bytes is NULL");
    qai_status s = check_window(window, stride);
    if (s != QAI_OK) return s;
    Shape sh;
    if ((s = make_shape(rank, dims, &sh)) != QAI_OK) return s;
    const qai::QualArgs a = quality_args(sh, window, stride);
    *bytes = quality_stat_bytes() + align256(sizeof(double) * (size_t)qai::quality_ssim_blocks(a));
    return QAI_OK;
}

qai_status qai_quality(const float* d_x, const float* d_y, int rank, const int64_t* dims, int window,
                       int stride, qai_quality_out* d_result, float* d_ssim_map, void* d_ws,
                       size_t ws_bytes, cudaStream_t stream)
{
    g_last_error.clear();
    if (!d_x || !d_y || !d_result) return fail(QAI_ERR_INVALID_ARG, "d_x, d_y and d_result must be non-NULL");
    size_t need = 0;
    qai_status s = qai_workspace_size_quality(rank, dims, window, stride, &need);
    if (s != QAI_OK) return s;
    if (!d_ws || ws_bytes < need)
        return fail(QAI_ERR_INVALID_ARG, "qai_quality needs a workspace of %zu bytes", need);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255) return fail(QAI_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    Shape sh;
    make_shape(rank, dims, &sh);
    qai::QualArgs a = quality_args(sh, window, stride);
    a.x = d_x;
    a.y = d_y;
    a.result = d_result;
    a.map = d_ssim_map;
    const int blocks = (int)std::min<int64_t>(kQualStatBlocks, (sh.N + 255) / 256);
    a.partials = static_cast<double*>(d_ws);
    cudaError_t e = timed("quality_stats", (double)sh.N * 8, stream,
                          [&] { return qai::launch_quality_stats(a, sh.N, blocks, stream); });
    count_launch();  // the one-block combine
    if (e != cudaSuccess) return cuda_fail(e, "quality stats");
    a.partials = reinterpret_cast<double*>(static_cast<char*>(d_ws) + quality_stat_bytes());
    e = timed("quality_ssim", (double)sh.N * 8, stream, [&] { return qai::launch_quality_ssim(a, stream); });
    count_launch();
    if (e != cudaSuccess) return cuda_fail(e, "quality ssim");
    return QAI_OK;
}

qai_status qai_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return QAI_OK;
}

qai_status qai_profile_select(const char* name)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_only = name ? name : "";
    return QAI_OK;
}

int qai_profile_read(qai_kernel_stat* out, int cap)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (const Pending& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            Stat* st = nullptr;
            for (Stat& s : g_stats)
                if (s.name == p.name) st = &s;
            if (!st) {
                g_stats.push_back(Stat{});
                st = &g_stats.back();
                st->name = p.name;
            }
            st->launches += 1;
            st->ms += ms;
            st->bytes += p.bytes;
        }
        g_event_pool.push_back(p.a);
        g_event_pool.push_back(p.b);
    }
    g_pending.clear();
    int n = 0;
    for (const Stat& s : g_stats) {
        if (n >= cap || !out) break;
        std::memset(&out[n], 0, sizeof(qai_kernel_stat));
        std::strncpy(out[n].name, s.name.c_str(), sizeof(out[n].name) - 1);
        out[n].launches = s.launches;
        out[n].total_ms = s.ms;
        out[n].algo_bytes = s.bytes;
        ++n;
    }
    g_stats.clear();
    return n;
}

int64_t qai_launch_count(void) { return g_launches.load(); }

const char* qai_status_string(qai_status s)
{
    switch (s) {
        case QAI_OK: return "QAI_OK";
        case QAI_ERR_INVALID_ARG: return "QAI_ERR_INVALID_ARG";
        case QAI_ERR_SHAPE: return "QAI_ERR_SHAPE";
        case QAI_ERR_RANGE: return "QAI_ERR_RANGE";
        case QAI_ERR_CUDA: return "QAI_ERR_CUDA";
        case QAI_ERR_OOM: return "QAI_ERR_OOM";
        case QAI_ERR_TIMEOUT: return "QAI_ERR_TIMEOUT";
        case QAI_ERR_INTERNAL: return "QAI_ERR_INTERNAL";
    }
    return "QAI_ERR_UNKNOWN";
}

const char* qai_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
