// qai_host.h -- host-side helpers shared by the C-ABI translation units
// (internal): shapes, workspace layout, parameter checks, error reporting.
#pragma once
#include <cstddef>
#include <cstdint>
#include <functional>
#include <cuda_runtime.h>

#include "qai.h"
#include "qai_device.cuh"
#include "qai_launch.h"

namespace qai {
namespace host {

// A field after squeezing extent-1 axes: rank 1..3, extents nz, ny, nx.
struct Shape {
    int rank;
    int nz, ny, nx;
    int64_t N;
};

// Byte offsets of the workspace slices of one field.
struct Layout {
    size_t eqm, xw, yw, dist1, s, idx, cflag;
    // signed-point route (rank 2 and 3): counters, queries, queries left to
    // the brute-force search, B2 sites; capacities in entries
    size_t ctr, qlist, slist, mlist, flist, fmin, b2list;
    // the local first EDT and the route: packed step-A codes, differ maps
    // and S (wpr words a row), the B2 bitmap (bwpr words a row)
    size_t codes, nexy, nez, spk, b2bits;
    int wpr, bwpr;
    int qcap, scap, fcap, b2cap;
    size_t total;
};

qai_status fail(qai_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
qai_status cuda_fail(cudaError_t e, const char* what);
qai_status make_shape(int rank, const int64_t* dims, Shape* s);
size_t align256(size_t v);
Layout layout_for(const Shape& s, uint32_t flags);
qai_status check_params(const qai_params* p);
MethodArgs method_args(const qai_params* p, double eb);
void count_launch();
// One launch through fn, counted and, while profiling, timed as kernel `name`
// with `algo_bytes` algorithmic bytes.
cudaError_t timed_call(const char* name, double algo_bytes, cudaStream_t st, const std::function<cudaError_t()>& fn);

// qai_mitigate's launch sequence without per-step outputs (a plain call) on a
// validated shape and a workspace laid out by layout_for(sh, 0).
qai_status run_plain(const int32_t* d_q, float* d_out, const Shape& sh, const MethodArgs& m, char* ws,
                     const Layout& lay, cudaStream_t st);

// The argument structs of a plain call's kernels on one rank-2 or rank-3
// field (step A, the local first EDT with its separable fallback, the
// signed-point route with the dense second EDT behind it), as run_plain
// launches them, for the batched form's grouped launches. The route counters
// live at `ctr`. Column passes: c1[0] / c2[0] along y, c1[1] / c2[1] along z
// (rank 3), prepared for the plain call's tiles (cfg1 / cfg2).
struct PlainArgs {
    LocalArgs la;
    RouteArgs ra;
    RowArgs r1, r2;
    ColArgs c1[2], c2[2];
    ColConfig cfg1[2], cfg2[2];
};
bool plain_args(const int32_t* d_q, float* d_out, const Shape& sh, const MethodArgs& m, char* ws,
                const Layout& lay, int* ctr, PlainArgs* pa);

// While alive, the library's launches on this host thread are counted into
// *counter and not timed or counted globally (launches recorded into a graph).
class LaunchSink {
public:
    explicit LaunchSink(int* counter);
    ~LaunchSink();
    LaunchSink(const LaunchSink&) = delete;
    LaunchSink& operator=(const LaunchSink&) = delete;

private:
    int* prev_;
};

}  // namespace host
}  // namespace qai
