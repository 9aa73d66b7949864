// qai_device.cuh -- encodings, argument blocks and device helpers shared by
// the qai CUDA kernels (row pass, column pass) and their host launchers.
//
// Pipeline of Algorithm 4 on a field of extents (nz, ny, nx), x contiguous:
//
//   row pass 1     step A (Algorithm 2) + first EDT pass along x on B1
//   column pass 1  EDT along y, then z (Algorithm 1), carrying the sign of
//                  the nearest boundary; the last pass writes Dist1 and S
//                  (step C's propagation, Algorithm 3, happens for free)
//   row pass 2     GetBoundary(S) -> B2 (Algorithm 3) + EDT pass along x
//   column pass 2  EDT along y, then z; the last pass fuses step E
//                  (IDW compensation) so Dist2 never reaches memory.
//
// Intermediate words (all-ones = "no site reached yet"):
//   xword  u16  phase 1: (d << 2) | sign code, d = |x - x_site| <= 16382
//               phase 2: d
//   yword  u32  phase 1: (g << 2) | sign code, g = dx^2 + dy^2 < 2^30
//               phase 2: g
// Sign code: 0 -> 0, 1 -> +1, 2 -> -1.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qai {

constexpr uint16_t kInf16 = 0xFFFFu;
constexpr uint32_t kInf32 = 0xFFFFFFFFu;
constexpr int32_t kDistInf = 0x7FFFFFFF;

__host__ __device__ inline int sign_code(int s) { return s > 0 ? 1 : (s < 0 ? 2 : 0); }
__host__ __device__ inline int sign_of_code(int c) { return c == 1 ? 1 : (c == 2 ? -1 : 0); }

struct MethodArgs {
    float two_eb;        // 2 eps, the dequantization step of Eq. 1
    float eta_eb;        // eta * eps, the boundary error magnitude of step E
    float idw_power;     // p of the inverse-distance weights
    int idw_is_one;      // p == 1 (the paper's weights): no powf
    int grad_threshold;  // Algorithm 2 fast-varying test, integer form
    int sign_rule;       // 0 SUM, 1 FIRST
    int b2_rule;         // 0 SAME_Q, 1 LITERAL
    int output_c;        // write the compensation C instead of D''
    unsigned flags;      // qai_params.flags (route selection bits)
};

// Programmatic dependent launch: a kernel launched by launch_chained (see
// qai_launch.h) may be scheduled while the kernel before it on the stream is
// still finishing; it waits here, before it reads or writes any memory, for
// that kernel to complete and its writes to be visible. Launched without the
// attribute, the wait returns at once.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Signed-point route of the second EDT (qai_signed.cu). Step E adds
// C = S w eta eps: where S = 0 the output is D' whatever Dist2 is, and on B1
// (Dist1 = 0) the weight is 1 whatever Dist2 is. Dist2 is needed only at the
// "queries": points with S != 0 off B1. The route counters live in the
// workspace; row pass 1 zeroes them.
enum RouteCtr : int {
    kCtrQueries = 0,   // queries appended (by near, or the last separable EDT1 pass)
    kCtrUnresolved = 1,// queries the shell search left to the search over the B2 sites
    kCtrB2 = 2,        // B2 sites listed for that search
    kCtrDense = 3,     // != 0: the dense second EDT must run
    kCtrSigned = 4,    // B1 points with S != 0
    kCtrSignedOver = 5,// != 0: the list of them is incomplete (a CTA had more than it could buffer)
    kCtrBruteDone = 6, // CTAs of the brute-force search that finished
    kCtrNearItems = 7, // items of the nearest-site search handed out (one-field launch)
    kCtrMid = 8,       // queries the first (per-thread) shell search left
    kCtrBitmap = 9,    // != 0: the bitmap route runs (the sparse route could not)
    kCtrWide = 12,     // != 0: an index outside the fast path's range: the exact step A ran
    kCtrSignedExact = 13, // B1 points with S != 0, counted by the exact step A
    kCtrTimeout = 14,  // != 0: a bounded device-side wait ran out (the call's output is not valid)
    kCtrLocalFail = 15,// != 0: the local first EDT left a point without its site;
                       // the separable first EDT runs (and zeroes the words before)
    kCtrWords = 16
};
// A query: linear index and (Dist1 << 2) | sign code of S.
struct Query {
    int32_t idx;
    int32_t d1code;
};

// Row pass: one warp per x-row; rows enumerated (z, y).
struct RowArgs {
    int rank, nz, ny, nx;
    int vec;                 // 128-bit access path usable (set by the launcher)
    const int32_t* q;        // phase 1 input; phase 2 final: D' source
    uint8_t* eqm;            // phase 1 writes, phase 2 reads: equal-q neighbour mask
    const int8_t* s_in;      // phase 2: propagated sign map S
    const int32_t* dist1_in; // phase 2 final (rank 1)
    uint16_t* xw;            // non-final output words
    int32_t* dist1;          // phase 1 final (rank 1)
    int8_t* s_out;           // phase 1 final (rank 1)
    float* out;              // phase 2 final (rank 1)
    // optional per-step outputs (NULL = skip)
    uint8_t* dbg_b1;
    int8_t* dbg_sb;
    int32_t* dbg_idx;        // phase 1: nearest-site linear index along the row
    uint8_t* dbg_b2;
    int32_t* dbg_dist2;      // phase 2 final (rank 1)
    // Signed-point route (rank 2 and 3, plain calls): phase 1 writes the
    // output at every point (D' + S_B eta eps on B1, D' elsewhere) and zeroes
    // the counters below kCtrLocalFail. gate: the kernel runs only when *gate
    // != 0 (then on a resident grid that loops over the rows).
    float* out_pre;
    int* route_ctr;
    const int* gate;
    MethodArgs m;
};

// Column pass over lines along one axis. Element (plane p, row r, column c)
// lives at p * plane_stride + r * row_stride + c for every array involved.
struct ColArgs {
    const void* in;          // xword (IN = 2) or yword (IN = 4) input
    int L;                   // line length (rows along the pass axis)
    int C;                   // columns per plane (contiguous)
    int P;                   // planes
    int64_t row_stride, plane_stride;
    int bands;               // B, rows are split in B bands of ceil(L / B)
    int load_bytes;          // cp.async width of the tile staging (16, 8, 4; 0 = plain loads)
    int narrow;              // RemoveEDT fits 32-bit arithmetic (set by the launcher)
    void* out_w;             // non-final output words (yword)
    int32_t* dist1;          // phase 1 final
    int8_t* s_out;           // phase 1 final
    float* out;              // phase 2 final
    const int32_t* q;        // phase 2 final
    const int32_t* dist1_in; // phase 2 final
    const int8_t* s_in;      // phase 2 final
    const int32_t* dbg_idx_in;   // phase 1: carried nearest-site index
    int32_t* dbg_idx_out;
    int32_t* dbg_dist2;      // phase 2 final
    const float* grad_out;   // phase 2 final, adjoint mode: dL/dD'' (no D'' written)
    double* partials;        // adjoint mode: two FP64 sums per CTA
    // Per column (index p * C + c), the number of points with S != 0
    // (saturated at 65535): written by the last pass of the first EDT, read by
    // the last pass of the second, which streams D'' = D' through tiles
    // without such points and scans for Dist2 only at them where they are few.
    uint16_t* col_count_out;
    const uint16_t* col_count_in;
    // Signed-point route (plain calls). Phase 1 final: Dist1 is written only
    // where S != 0 and each query is appended to qlist (at most qcap; the
    // count goes on past it); phase 2 final writes only points with S != 0
    // (the first EDT wrote every other output). gate: the pass runs only when
    // *gate != 0 (then on a resident grid that loops over the tiles).
    int* route_ctr;
    const int* gate;
    // Phase 2 final after the local first EDT: Dist1 is not stored on B1;
    // a point is on B1 where its equal-q mask byte has a clear bit, and its
    // Dist1 is 0 there.
    const uint8_t* b1_eqm;
    int32_t* d2rec;          // phase 2 final in the route: NULL, or Dist2 recorded at S != 0
    Query* qlist;
    int qcap;
    int32_t* slist;          // B1 points with S != 0 (linear indices), at most scap
    int scap;
    MethodArgs m;
};

// The kernels of the signed-point route.
struct RouteArgs {
    int rank, nz, ny, nx;
    int wpr, bwpr;           // packed words per row: S (16 points), B2 bitmap (32)
    const int32_t* q;
    const uint32_t* spk;     // packed S
    const uint32_t* nexy;    // packed differ maps of step A
    const uint32_t* nez;
    uint32_t* b2bits;        // B2 bitmap (written by k_b2map)
    float* out;
    int* ctr;                // RouteCtr words
    const Query* qlist;
    int qcap;
    const int32_t* slist;    // B1 points with S != 0 (the rest of the signed set), at most scap
    int scap;
    Query* mlist;            // queries left by the first shell search (qcap entries)
    Query* flist;            // queries left to the brute-force search
    int32_t* fmin;           // their Dist2, min-reduced by the brute-force CTAs
    int fcap;
    int32_t* b2list;         // B2 sites as (x | y << 16, z) pairs
    int b2cap;
    int32_t* d2rec;          // NULL, or Dist2 recorded here (by point) at every query
    int shell;               // 0: no shell search (every query to the site list)
    long long brute_budget;  // largest leftover queries x sites product searched by brute force
    MethodArgs m;
};

// The local first EDT (qai_local.cu): step A, then the nearest B1 site of
// every point by a bounded exact search, S and the signed-point lists.
//
// Packed per-point maps (2 bits a point, 16 points a 32-bit word; each row
// of x starts a new word, so a row takes wpr = ceil(nx / 16) words and the
// fields past nx are 0): point (row, x) is field x & 15 of word
// row * wpr + (x >> 4), at bits 2 (x & 15) and up.
//   codes  step A: 0 off B1, 1 + sign code of S_B on B1 (1: S_B = 0,
//          2: S_B = +1, 3: S_B = -1)
//   nexy   q != q[x + 1] (low bit) and q != q[y + 1] (high bit) of each
//          point (not defined where the neighbour does not exist)
//   nez    q != q[z + 1] (low bit; rank 3)
//   spk    S (Algorithm 3) as a sign code: 0, 1 (+1), 2 (-1)
// The B2 bitmap of the route is 1 bit a point, 32 points a word, a row
// taking bwpr = ceil(nx / 32) words (bits past nx are 0).
struct LocalArgs {
    int rank, nz, ny, nx;
    int wpr;                 // packed words per row
    const int32_t* q;
    uint32_t* codes;         // packed step-A codes (written by detect)
    uint32_t* nexy;          // packed q != q[x + 1] (low bit), q != q[y + 1] (high bit)
    uint32_t* nez;           // packed q != q[z + 1] (low bit; rank 3)
    uint32_t* spk;           // packed S (written by near)
    int32_t* dist1;          // Dist1 at the queries (S != 0 off B1)
    float* out;              // D' + S_B eta eps on B1, D' elsewhere
    int* ctr;                // RouteCtr words
    Query* qlist;
    int qcap;
    int32_t* slist;          // B1 points with S != 0 (linear indices), at most scap
    int scap;
    int vec;                 // 128-bit loads of q usable
    // the byte maps of the separable passes, for the fallbacks: eqm (equal-q
    // mask, bits 0-5, and the sign code of S_B, bits 6-7; 0x3F off the
    // interior) and s (S as int8)
    uint8_t* eqm;
    int8_t* s;
    MethodArgs m;
    int near_stride;         // one-field near launch: the t-th item taken is t * near_stride mod items
};

// Grouped launches: several fields in one kernel, the per-field arguments
// passed by value in the kernel parameters (at most kMaxGroup per launch).
constexpr int kMaxGroup = 96;
struct RowTable {
    int n;
    int warps;                        // warps per CTA
    int smem_nx;                      // x extent the per-warp shared memory is sized for
    int first_row[kMaxGroup + 1];     // row offsets; first_row[n] = rows in total
    RowArgs args[kMaxGroup];
};

// Persistent grouped launches (the batched form): one launch runs one
// kernel body over several fields. Field f gets vb[f] virtual blocks (the
// grid it would get alone, or a share of it); a field whose gate reads 0 when
// the launch starts gets none (the gates are flags that earlier launches set
// and no body of this launch changes). The resident CTAs take virtual blocks
// from a device cursor, in field order, until none is left, and run the body
// with the field's arguments (a device array) and the virtual block index and
// count in place of blockIdx.x and gridDim.x. The bodies do not depend on
// which CTA runs a virtual block, nor on a field's virtual blocks running at
// the same time.
constexpr int kGroupMax = 64;
struct GroupQueue {
    int n;                         // fields
    int* cursor;                   // next virtual block (zeroed before the launch)
    const void* args;              // the fields' argument structs, device memory
    int vb[kGroupMax];             // virtual blocks of each field
    const int* gate[kGroupMax];    // NULL, or the field runs only if *gate != 0
};

template <class Args, class Body>
__device__ __forceinline__ void run_group(const GroupQueue& q, Body&& body)
{
    __shared__ int s_first[kGroupMax + 1];
    __shared__ int s_item;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    wait_prior_grid();  // the gates and the fields' inputs come from earlier launches
    for (int f = tid; f < q.n; f += nthr)
        s_first[f + 1] = (!q.gate[f] || *static_cast<const volatile int*>(q.gate[f]) != 0) ? q.vb[f] : 0;
    __syncthreads();
    if (tid == 0) {
        s_first[0] = 0;
        for (int f = 1; f <= q.n; ++f) s_first[f] += s_first[f - 1];
    }
    __syncthreads();
    const int total = s_first[q.n];
    for (;;) {
        if (tid == 0) s_item = total > 0 ? atomicAdd(q.cursor, 1) : total;
        __syncthreads();
        const int it = s_item;
        __syncthreads();  // s_item is read before the next item overwrites it
        if (it >= total) return;
        int lo = 0, hi = q.n - 1;  // the last field starting at or before it (never an empty one)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_first[mid] <= it) lo = mid;
            else hi = mid - 1;
        }
        const Args a = static_cast<const Args*>(q.args)[lo];
        body(a, it - s_first[lo], s_first[lo + 1] - s_first[lo]);
    }
}

// A float-float value hi + lo: the sum of two of them keeps the rounding
// error of hi + hi' exactly (Knuth's two-sum), so a tree of such sums loses
// no more than a few units of 2^-44 of its magnitude without FP64 work.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float hi2, float lo2)
{
    const float s = hi + hi2;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (hi2 - bp);
    const float l = lo + lo2 + e;
    hi = s + l;
    lo = l - (hi - s);
}

// Per-thread sums of the adjoint terms: fp32 with Kahan compensation, taken
// to FP64 once by fold() (the error stays below 2 eps32 of the sum of |term|
// for the few thousand terms one thread adds). No FP64 work in the loop: a
// periodic fold would be predicated onto every term, and the FP64 pipe is
// narrow.
struct GradAcc {
    float se = 0.f, ce = 0.f, sp = 0.f, cp = 0.f;
    double de = 0.0, dp = 0.0;
    __device__ __forceinline__ void add(float te, float tp)
    {
        float y = te - ce, t = se + y;
        ce = (t - se) - y;
        se = t;
        y = tp - cp;
        t = sp + y;
        cp = (t - sp) - y;
        sp = t;
    }
    __device__ __forceinline__ void fold()
    {
        de += (double)se - (double)ce;
        dp += (double)sp - (double)cp;
        se = ce = sp = cp = 0.f;
    }
};

// Adjoint of step E: a reduction over the points (qai_backward.cu).
constexpr int kBackwardMaxBlocks = 2048;
struct BackArgs {
    int64_t N;
    const float* grad_out;   // dL/dD''
    const int8_t* s;         // S
    const int32_t* dist1;    // Dist1 (read only where S != 0)
    const int32_t* dist2;    // Dist2 (idem)
    const uint8_t* b1_eqm;   // NULL, or equal-q mask bytes: Dist1 = 0 where a bit is clear (B1)
    // or, after a plain forward: S and B1 from its packed maps (s and b1_eqm
    // unused): S from spk, B1 where the step-A code is not 0 (wpr words a row)
    const uint32_t* spk;
    const uint32_t* codes;
    int wpr, nx;
    float* grad_dprime;      // dL/dD' (= dL/dD''), NULL to skip
    double* grad_params;     // [2]: dL/deta, dL/dp
    double* partials;        // [2 * kBackwardMaxBlocks] block totals (workspace)
    float p;                 // IDW exponent
    double eta, eb;
};

// PTX approximate square root, reciprocal, log2 and exp2 (a few ulp each;
// the weights they feed are compared at 1e-6 of the value range).
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Step E for one point: C = S * w * eta * eps with the inverse-distance weight
// w = k2^p / (k1^p + k2^p) of the distances k1 = sqrt(Dist1), k2 = sqrt(Dist2);
// a point on B1 gets w = 1 (this takes precedence), a point on B2 gets w = 0,
// and a field without B2 gives w = 1 (the limit k2 -> infinity).
// For p = 1, w = k2 / (k1 + k2) = Dist2 / (sqrt(Dist1 Dist2) + Dist2); for
// other p, w = 1 / (1 + 2^(p/2 (log2 Dist1 - log2 Dist2))). No branches: the
// special cases are selects, and S = 0 zeroes C through the product.
__device__ __forceinline__ float compensate(int32_t q, int32_t d1, int32_t d2, int s,
                                            const MethodArgs& m)
{
    const float f1 = (float)d1, f2 = (float)d2;
    float w;
    if (m.idw_is_one) {
        w = f2 * rcp_approx(sqrt_approx(f1 * f2) + f2);
    } else {
        const float t = ex2_approx(0.5f * m.idw_power * (lg2_approx(f1) - lg2_approx(f2)));
        w = rcp_approx(1.0f + t);
    }
    w = d2 == kDistInf ? 1.0f : w;
    w = d2 == 0 ? 0.0f : w;
    w = d1 == 0 ? 1.0f : w;
    const float fs = s > 0 ? 1.0f : (s < 0 ? -1.0f : 0.0f);
    const float c = fs * w * m.eta_eb;
    return m.output_c ? c : fmaf((float)q, m.two_eb, c);
}

// The two summands of the adjoint of step E at one point, before the factors
// eb (dL/deta) and eta * eb (dL/dp): te = G S w, tp = G S dw/dp, with
// (k1/k2)^p = 2^(p/2 log2(d1/d2)) and dw/dp = -w (1 - w) ln(k1/k2). The log
// is taken of the ratio, so points with d1 close to d2 lose no digits; dw/dp
// is 0 where w is pinned (k1 = 0, k2 = 0, no B2).
__device__ __forceinline__ void grad_terms(float g, int s, int32_t d1, int32_t d2, float p,
                                           float& te, float& tp)
{
    const float l = lg2_approx((float)d1 * rcp_approx((float)d2));  // log2(d1 / d2)
    const float t = ex2_approx(0.5f * p * l);
    float w = rcp_approx(1.0f + t);
    float dw = w * (1.0f - w) * (-0.5f * 0.69314718f) * l;
    const bool pinned = d1 == 0 || d2 == 0 || d2 == kDistInf;
    w = d2 == kDistInf ? 1.0f : w;
    w = d2 == 0 ? 0.0f : w;
    w = d1 == 0 ? 1.0f : w;
    dw = pinned ? 0.0f : dw;
    // S = 0: no term, whatever d1 and d2 hold (they need not be written there)
    const float gs = s > 0 ? g : -g;
    te = s ? gs * w : 0.0f;
    tp = s ? gs * dw : 0.0f;
}

}  // namespace qai
