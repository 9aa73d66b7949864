// qai_signed.cu -- the signed-point route of the second EDT (step D) and of
// step E.
//
// Step E adds C = S w eta eps (Sec. VI-E). Where S = 0 the output is D'
// whatever Dist2 is, and on B1 (Dist1 = 0) the weight is 1 whatever Dist2 is
// (the boundary value eta eps); row pass 1 writes both of these outputs. Dist2
// is needed only at the queries -- points with S != 0 off B1 -- which the last
// pass of the first EDT lists, with the B1 points that have S != 0. These
// kernels then give the exact Dist2 of every query, Eq. 2 over the
// sign-flipping boundary B2 of Algorithm 3:
//
//   k_query    a shell search around the query (one thread each, then one
//              warp, then one CTA each for the queries the phase before
//              left): lattice offsets in order of squared length,
//              GetBoundary(S) evaluated at each candidate from S and the
//              equal-q mask; the first hit is the minimum. A query with no B2
//              site within the search radius is left to the brute-force
//              search.
//   k_b2sites  (only when such queries exist) lists the B2 sites from the
//              signed points and their axis neighbours, or, when the list of
//              signed points overflowed, from a pass over the whole field;
//   k_brute    (idem) min over the site list for each remaining query.
//
// A count over a capacity, or a brute-force product over its budget, sets the
// dense flag; the dense second EDT (row pass 2, column passes 2) runs only
// then, and rewrites every point with S != 0. Every route gives the same bits:
// the same Dist2 goes into the same compensate().
#include "qai_device.cuh"
#include "qai_launch.h"

namespace qai {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Lattice offsets in order of squared length, then (dz, dy, dx):
// (r2 << 24) | (dz & 0xFF) << 16 | (dy & 0xFF) << 8 | (dx & 0xFF), so r2 <=
// 255. off3 spans three axes up to squared length kTableR2 (radius 6), off2
// two axes (dz = 0) up to kTableR2_2 (radius 15.9); the search phases take
// at most 1184 offsets (160 by a warp, 1024 by a CTA).
constexpr int kTableR2 = 36;
constexpr int kTableR = 6;
constexpr int kTableR2_2 = 255;
constexpr int kTableR_2 = 15;
constexpr int kN3 = 925, kN2 = 793;
struct OffsetTable {
    int off3[kN3];
    int off2[kN2];
};
constexpr int pack_offset(int r2, int dz, int dy, int dx)
{
    return (int)(((unsigned)r2 << 24) | ((unsigned)(dz & 0xFF) << 16) | ((unsigned)(dy & 0xFF) << 8) |
                 (unsigned)(dx & 0xFF));
}
constexpr int isqrt_c(int v)
{
    int r = 0;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}
constexpr OffsetTable make_offsets()
{
    OffsetTable t{};
    int n3 = 0, n2 = 0;
    for (int r2 = 0; r2 <= kTableR2; ++r2)
        for (int dz = -kTableR; dz <= kTableR; ++dz)
            for (int dy = -kTableR; dy <= kTableR; ++dy)
                for (int dx = -kTableR; dx <= kTableR; ++dx)
                    if (dz * dz + dy * dy + dx * dx == r2) t.off3[n3++] = pack_offset(r2, dz, dy, dx);
    for (int r2 = 0; r2 <= kTableR2_2; ++r2)
        for (int dy = -kTableR_2; dy <= kTableR_2; ++dy) {
            const int rest = r2 - dy * dy;
            if (rest < 0) continue;
            const int dx = isqrt_c(rest);
            if (dx * dx != rest) continue;
            t.off2[n2++] = pack_offset(r2, 0, dy, -dx);  // increasing dx
            if (dx > 0) t.off2[n2++] = pack_offset(r2, 0, dy, dx);
        }
    return t;
}
// the tables hold exactly kN3 and kN2 offsets
constexpr int count_offsets(int r2max, int r, bool three)
{
    int n = 0;
    for (int dz = three ? -r : 0; dz <= (three ? r : 0); ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                if (dz * dz + dy * dy + dx * dx <= r2max) ++n;
    return n;
}
static_assert(count_offsets(kTableR2, kTableR, true) == kN3, "3-D offset table size");
static_assert(count_offsets(kTableR2_2, kTableR_2, false) == kN2, "2-D offset table size");
static_assert(kTableR2_2 <= 255 && (kTableR_2 + 1) * (kTableR_2 + 1) > kTableR2_2, "2-D table radius");
__constant__ OffsetTable c_off = make_offsets();

// GetBoundary(S) of Algorithm 3 at an interior point b: an axis neighbour
// (with the same q, under the SAME_Q reading) has a different S.
// Every load is issued before any test, so their latencies overlap.
template <int RANK>
__device__ __forceinline__ bool is_b2(const RouteArgs& a, int64_t b)
{
    const int64_t pl = (int64_t)a.ny * a.nx;
    const int sb = __ldg(a.s + b);
    const unsigned em = a.m.b2_rule == 1 ? 0x3Fu : (unsigned)__ldg(a.eqm + b);
    const int xl = __ldg(a.s + b - 1), xr = __ldg(a.s + b + 1);
    const int yl = __ldg(a.s + b - a.nx), yr = __ldg(a.s + b + a.nx);
    const int zl = RANK == 3 ? __ldg(a.s + b - pl) : sb, zr = RANK == 3 ? __ldg(a.s + b + pl) : sb;
    const unsigned diff = (unsigned)(zl != sb) | (unsigned)(zr != sb) << 1 | (unsigned)(yl != sb) << 2 |
                          (unsigned)(yr != sb) << 3 | (unsigned)(xl != sb) << 4 | (unsigned)(xr != sb) << 5;
    return (diff & em) != 0;
}

__device__ __forceinline__ float query_output(const RouteArgs& a, const Query& e, int32_t d2)
{
    return compensate(__ldg(a.q + e.idx), e.d1code >> 2, d2, sign_of_code(e.d1code & 3), a.m);
}

// The output of a query with its Dist2 (recorded too when asked).
__device__ __forceinline__ void emit_query(const RouteArgs& a, const Query& e, int32_t d2)
{
    a.out[e.idx] = query_output(a, e, d2);
    if (a.d2rec) a.d2rec[e.idx] = d2;
}

// Offset k of the table at query (x, y, z): a B2 site? r2 = its squared
// length (r2 > max_r2, or k past the table: no).
template <int RANK>
__device__ __forceinline__ bool probe(const RouteArgs& a, int x, int y, int z, int k, int& r2)
{
    const int* tab = RANK == 3 ? c_off.off3 : c_off.off2;
    constexpr int ntab = RANK == 3 ? kN3 : kN2;
    const int o = k < ntab ? tab[k] : -1;
    r2 = (int)((unsigned)o >> 24);
    if (k >= ntab || r2 > a.max_r2) return false;
    const int bx = x + (int)(int8_t)(o & 0xFF);
    const int by = y + (int)(int8_t)((o >> 8) & 0xFF);
    const int bz = z + (int)(int8_t)((o >> 16) & 0xFF);
    // B2 lies on interior points only (extents of kept axes are >= 2)
    const bool inner = (unsigned)(bx - 1) < (unsigned)(a.nx - 2) && (unsigned)(by - 1) < (unsigned)(a.ny - 2) &&
                       (RANK == 2 || (unsigned)(bz - 1) < (unsigned)(a.nz - 2));
    return inner && is_b2<RANK>(a, (int64_t)bz * a.ny * a.nx + (int64_t)by * a.nx + bx);
}

__device__ __forceinline__ void coords(const RouteArgs& a, int idx, int& x, int& y, int& z)
{
    const int plane = a.ny * a.nx;
    z = idx / plane;
    const int rem = idx - z * plane;
    y = rem / a.nx;
    x = rem - y * a.nx;
}

// The shell search runs in three phases, each on the queries the one before
// left: one thread per query over the offsets of squared length 0 and 1
// (most queries end there), one warp per query over the offsets up to
// kPhase1, one CTA per query over the rest of the table. The first hit in
// table order has the smallest squared distance (the table is sorted by it).
constexpr int kPhase1 = 160;
static_assert(7 + 32 <= kPhase1, "the first round of the second phase lies inside it");
constexpr int kMidBuf = 2048;  // per-CTA buffer of the first phase's leftovers

// The first phase for a query p at least two steps inside every kept axis:
// 0 if p is a B2 site, else 1 if one of its axis neighbours is, else -1 --
// the offsets of squared length 0 and 1 in table order, read off the 25 S
// values (13 in 2-D) around p, each loaded once, and the seven mask bytes.
template <int RANK>
__device__ __forceinline__ int near_b2(const RouteArgs& a, int64_t p)
{
    const int64_t X = 1, Y = a.nx, Z = (int64_t)a.ny * a.nx;
    const int64_t st[6] = {-Z, Z, -Y, Y, -X, X};  // mask bit order z-, z+, y-, y+, x-, x+
    const bool literal = a.m.b2_rule == 1;
    auto has = [](int k) { return RANK == 3 || k >= 2; };
    const int sc = __ldg(a.s + p);
    int sn[6];
    unsigned en[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        sn[k] = has(k) ? (int)__ldg(a.s + p + st[k]) : sc;
        en[k] = has(k) && !literal ? (unsigned)__ldg(a.eqm + p + st[k]) : 0x3Fu;
    }
    const unsigned ec = literal ? 0x3Fu : (unsigned)__ldg(a.eqm + p);
    // S two steps away along an axis, and one step along each of two axes
    int s2[6], sd[6][6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        s2[k] = has(k) ? (int)__ldg(a.s + p + 2 * st[k]) : 0;
#pragma unroll
        for (int j = 0; j < 6; ++j)
            sd[k][j] = has(k) && has(j) && (j >> 1) != (k >> 1) && j > k ? (int)__ldg(a.s + p + st[k] + st[j]) : 0;
    }
    unsigned d0 = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) d0 |= (unsigned)(sn[k] != sc) << k;
    if (d0 & ec) return 0;
    bool hit1 = false;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (!has(k)) continue;
        // the neighbours of p + st[k]: p + 2 st[k], p itself, p + st[k] + st[j]
        unsigned dk = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            if (!has(j)) continue;
            const int v = j == k ? s2[k] : (j == (k ^ 1) ? sc : (j > k ? sd[k][j] : sd[j][k]));
            dk |= (unsigned)(v != sn[k]) << j;
        }
        hit1 |= (dk & en[k]) != 0;
    }
    return hit1 ? 1 : -1;
}

template <int RANK>
__global__ void __launch_bounds__(256) k_query(RouteArgs a)
{
    wait_prior_grid();
    volatile int* ctr = a.ctr;
    if (ctr[kCtrDense]) return;
    const int nq = ctr[kCtrQueries];
    if (nq > a.qcap) {  // the list is incomplete: the dense route takes over
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr[kCtrDense] = 1;
        return;
    }
    constexpr int n0 = RANK == 3 ? 7 : 5;  // offsets of squared length 0 and 1
    __shared__ Query mbuf[kMidBuf];
    __shared__ int mn, mbase;
    if (threadIdx.x == 0) mn = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
        const Query e = a.qlist[i];
        int x, y, z;
        coords(a, e.idx, x, y, z);
        int found = -1;
        const bool deep = a.max_r2 >= 1 && x >= 2 && x <= a.nx - 3 && y >= 2 && y <= a.ny - 3 &&
                          (RANK == 2 || (z >= 2 && z <= a.nz - 3));
        if (deep) {
            found = near_b2<RANK>(a, e.idx);
        } else {
            bool hit[n0];
            int r2[n0];
#pragma unroll
            for (int k = 0; k < n0; ++k) hit[k] = probe<RANK>(a, x, y, z, k, r2[k]);
#pragma unroll
            for (int k = n0 - 1; k >= 0; --k)
                if (hit[k]) found = r2[k];
        }
        if (found >= 0) {
            emit_query(a, e, found);
        } else {
            const int k = atomicAdd(&mn, 1);
            if (k < kMidBuf) {
                mbuf[k] = e;
            } else {
                const int g = atomicAdd(a.ctr + kCtrMid, 1);
                if (g < a.qcap) a.mlist[g] = e;
            }
        }
    }
    __syncthreads();
    const int n = min(mn, kMidBuf);
    if (threadIdx.x == 0) mbase = n > 0 ? atomicAdd(a.ctr + kCtrMid, n) : 0;
    __syncthreads();
    for (int j = threadIdx.x; j < n && mbase + j < a.qcap; j += blockDim.x) a.mlist[mbase + j] = mbuf[j];
}

// Second phase: one warp per query, table offsets n0 .. kPhase1: first the
// 32 nearest (where most of these queries end), then the other four per lane
// with their loads in flight together.
template <int RANK>
__global__ void __launch_bounds__(256) k_query_mid(RouteArgs a)
{
    wait_prior_grid();
    volatile int* ctr = a.ctr;
    if (ctr[kCtrDense]) return;
    const int nm = min((int)ctr[kCtrMid], a.qcap);  // at most the queries
    constexpr int n0 = RANK == 3 ? 7 : 5;
    const int lane = threadIdx.x & 31;
    const int wstride = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nm; i += wstride) {
        const Query e = a.mlist[i];
        int x, y, z;
        coords(a, e.idx, x, y, z);
        int found = -1;
        int r2[5];
        bool hit[5];
        hit[0] = probe<RANK>(a, x, y, z, n0 + lane, r2[0]);  // n0 + 31 < kPhase1
        const unsigned h0 = __ballot_sync(kFull, hit[0]);
        if (h0) {
            found = __shfl_sync(kFull, r2[0], __ffs(h0) - 1);
        } else {
#pragma unroll
            for (int u = 1; u < 5; ++u) {
                const int k = n0 + 32 * u + lane;
                hit[u] = k < kPhase1 && probe<RANK>(a, x, y, z, k, r2[u]);
            }
#pragma unroll
            for (int u = 1; u < 5; ++u) {
                const unsigned h = __ballot_sync(kFull, hit[u]);
                if (h && found < 0) found = __shfl_sync(kFull, r2[u], __ffs(h) - 1);
            }
        }
        if (lane == 0) {
            if (found >= 0) {
                emit_query(a, e, found);
            } else {
                const int k = atomicAdd(a.ctr + kCtrFailed, 1);
                if (k < a.fcap) {
                    a.flist[k] = e;
                    a.fmin[k] = kDistInf;
                }
            }
        }
    }
}

// Third phase: one CTA per query the second left, over table offsets
// kPhase1 .. (4 per thread: 1024 cover the 3-D table). A hit writes the
// output and marks the query done (fmin = -1); a miss leaves it to the
// brute-force search.
template <int RANK>
__global__ void __launch_bounds__(256) k_query_far(RouteArgs a)
{
    wait_prior_grid();
    volatile int* ctr = a.ctr;
    if (ctr[kCtrDense]) return;
    const int nf = ctr[kCtrFailed];
    if (nf > a.fcap) {  // the list is incomplete: the dense route takes over
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr[kCtrDense] = 1;
        return;
    }
    __shared__ int sbest[8];
    for (int f = blockIdx.x; f < nf; f += gridDim.x) {
        const Query e = a.flist[f];
        int x, y, z;
        coords(a, e.idx, x, y, z);
        int best = 0x7FFFFFFF;  // smallest table index with a hit
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = kPhase1 + (int)threadIdx.x + (int)blockDim.x * u;
            int r2;
            if (probe<RANK>(a, x, y, z, k, r2)) best = min(best, k);
        }
        best = __reduce_min_sync(kFull, best);
        if ((threadIdx.x & 31) == 0) sbest[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = min(best, sbest[w]);
            if (best != 0x7FFFFFFF) {
                const int* tab = RANK == 3 ? c_off.off3 : c_off.off2;
                emit_query(a, e, (int)((unsigned)tab[best] >> 24));
                a.fmin[f] = -1;
            } else {
                atomicAdd(a.ctr + kCtrUnresolved, 1);
            }
        }
        __syncthreads();
    }
}

// B2 sites found by one CTA, flushed to the global list with one atomic.
constexpr int kSiteBuf = 1024;
struct SiteBuf {
    uint2* e;  // [kSiteBuf] in shared memory
    int* n;    // shared count
};

// Appends the B2 sites x0 + j (bit j of nib) of row (y, z): into the CTA's
// buffer (warp-aggregated), or, when it is full, to the global list.
__device__ __forceinline__ void append_sites(const RouteArgs& a, const SiteBuf& sb, unsigned nib, int x0, int y, int z)
{
    const int lane = threadIdx.x & 31;
    if (!__ballot_sync(kFull, nib != 0)) return;
    const int cnt = __popc(nib);
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += v;
    }
    int base = 0;
    bool global = false;
    if (lane == 31) {
        base = atomicAdd(sb.n, incl);
        if (base + incl > kSiteBuf) {
            global = true;
            base = atomicAdd(a.ctr + kCtrB2, incl);
        }
    }
    global = __shfl_sync(kFull, global, 31);
    base = __shfl_sync(kFull, base, 31) + incl - cnt;
    uint2* list = global ? reinterpret_cast<uint2*>(a.b2list) : sb.e;
    const int cap = global ? a.b2cap : kSiteBuf;
    for (int j = 0; j < 4; ++j) {
        if (!((nib >> j) & 1u)) continue;
        if (base < cap) list[base] = make_uint2((uint32_t)(x0 + j) | ((uint32_t)y << 16), (uint32_t)z);
        ++base;
    }
}

__device__ __forceinline__ void flush_sites(const RouteArgs& a, const SiteBuf& sb, int* sbase)
{
    __syncthreads();
    const int n = min(*sb.n, kSiteBuf);
    if (threadIdx.x == 0) *sbase = n > 0 ? atomicAdd(a.ctr + kCtrB2, n) : 0;
    __syncthreads();
    uint2* list = reinterpret_cast<uint2*>(a.b2list);
    for (int i = threadIdx.x; i < n && *sbase + i < a.b2cap; i += blockDim.x) list[*sbase + i] = sb.e[i];
}

// The B2 sites, from the signed set: a site has S != 0 or an axis neighbour
// with S != 0 (GetBoundary(S) compares S across a pair), so every site is a
// signed point or an axis neighbour of one. Each signed point tests itself and
// its neighbours with S = 0; a neighbour with S = 0 is tested only by its
// signed neighbour of smallest linear index, so no site is listed twice.
// Runs when some query needs the list and the signed set is complete.
template <int RANK>
__device__ __forceinline__ void b2_from_field(const RouteArgs& a, const SiteBuf& sb, int vec);

template <int RANK>
__global__ void __launch_bounds__(256) k_b2sites(RouteArgs a, int vec)
{
    wait_prior_grid();
    volatile int* ctr = a.ctr;
    if (ctr[kCtrDense] || ctr[kCtrUnresolved] == 0) return;
    __shared__ uint2 sbuf[kSiteBuf];
    __shared__ int sn, sbase;
    if (threadIdx.x == 0) sn = 0;
    __syncthreads();
    const SiteBuf sb{sbuf, &sn};
    if (ctr[kCtrSignedOver] || ctr[kCtrSigned] > a.scap) {  // the signed set overflowed its list
        b2_from_field<RANK>(a, sb, vec);
        flush_sites(a, sb, &sbase);
        return;
    }
    const int ns = ctr[kCtrSigned], nq = ctr[kCtrQueries];
    const int plane = a.ny * a.nx;
    // one thread per signed point p: its candidates are p and its axis
    // neighbours, and every S they need lies within two axis steps of p, so
    // all loads of the thread are issued together
    for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < ns + nq; item += gridDim.x * blockDim.x) {
        const int p = item < ns ? a.slist[item] : a.qlist[item - ns].idx;
        int x, y, z;
        coords(a, p, x, y, z);
        // S at p + (dz, dy, dx), 0 outside the field (never read there: only
        // interior candidates are tested, and their neighbours lie inside)
        auto S = [&](int dz, int dy, int dx) -> int {
            const bool in = (unsigned)(x + dx) < (unsigned)a.nx && (unsigned)(y + dy) < (unsigned)a.ny &&
                            (RANK == 2 || (unsigned)(z + dz) < (unsigned)a.nz);
            return in ? (int)__ldg(a.s + p + dz * plane + dy * a.nx + dx) : 0;
        };
        // candidate c: 0 = p, then z-, z+, y-, y+, x-, x+ (rank 2: y-, y+, x-, x+)
#pragma unroll
        for (int c = 0; c <= 2 * RANK; ++c) {
            int cz = 0, cy = 0, cx = 0;
            if (c > 0) {
                const int ax = RANK == 3 ? (c - 1) >> 1 : ((c - 1) >> 1) + 1;
                const int sg = (c - 1) & 1 ? 1 : -1;
                (ax == 0 ? cz : (ax == 1 ? cy : cx)) = sg;
            }
            const int bx = x + cx, by = y + cy, bz = z + cz;
            const bool inner = (unsigned)(bx - 1) < (unsigned)(a.nx - 2) && (unsigned)(by - 1) < (unsigned)(a.ny - 2) &&
                               (RANK == 2 || (unsigned)(bz - 1) < (unsigned)(a.nz - 2));
            if (!inner) continue;
            const int sb0 = S(cz, cy, cx);
            // the six axis neighbours of the candidate: z-, z+, y-, y+, x-, x+
            int nbv[6];
            nbv[0] = RANK == 3 ? S(cz - 1, cy, cx) : sb0;
            nbv[1] = RANK == 3 ? S(cz + 1, cy, cx) : sb0;
            nbv[2] = S(cz, cy - 1, cx);
            nbv[3] = S(cz, cy + 1, cx);
            nbv[4] = S(cz, cy, cx - 1);
            nbv[5] = S(cz, cy, cx + 1);
            bool own = true;
            if (c > 0) {
                // an S = 0 candidate is tested by its signed neighbour of
                // smallest linear index: p must precede every other one (an
                // offset precedes 0 in (dz, dy, dx) order exactly when its
                // point precedes p, for points inside the field)
                own = sb0 == 0;
                const int oz[6] = {cz - 1, cz + 1, cz, cz, cz, cz}, oy[6] = {cy, cy, cy - 1, cy + 1, cy, cy},
                          ox[6] = {cx, cx, cx, cx, cx - 1, cx + 1};
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const bool before = oz[k] < 0 || (oz[k] == 0 && (oy[k] < 0 || (oy[k] == 0 && ox[k] < 0)));
                    if (before && nbv[k] != 0) own = false;
                }
            }
            if (!own) continue;
            const unsigned em = a.m.b2_rule == 1 ? 0x3Fu
                                                 : (unsigned)__ldg(a.eqm + p + cz * plane + cy * a.nx + cx);
            unsigned diff = 0;
#pragma unroll
            for (int k = 0; k < 6; ++k) diff |= (unsigned)(nbv[k] != sb0) << k;
            if (diff & em) {
                const int kk = atomicAdd(sb.n, 1);
                const uint2 e = make_uint2((uint32_t)bx | ((uint32_t)by << 16), (uint32_t)bz);
                if (kk < kSiteBuf) {
                    sb.e[kk] = e;
                } else {
                    const int g = atomicAdd(a.ctr + kCtrB2, 1);
                    if (g < a.b2cap) reinterpret_cast<uint2*>(a.b2list)[g] = e;
                }
            }
        }
    }
    flush_sites(a, sb, &sbase);
}

__device__ __forceinline__ uint32_t load4_s8(const int8_t* p, int x0, int nx, bool vec)
{
    if (vec) return x0 < nx ? __ldg(reinterpret_cast<const uint32_t*>(p + x0)) : 0u;
    uint32_t w = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (x0 + j < nx) w |= (uint32_t)(uint8_t)__ldg(p + x0 + j) << (8 * j);
    return w;
}

// Every B2 site of the field, for the case where the signed set overflowed
// its list. One warp per interior row, 128 points per step (4 per lane).
template <int RANK>
__device__ __forceinline__ void b2_from_field(const RouteArgs& a, const SiteBuf& sb, int vec)
{
    const int lane = threadIdx.x & 31;
    const int rows = a.nz * a.ny;
    const int plane = a.ny * a.nx;
    const uint8_t* eqm = a.eqm;
    const bool literal = a.m.b2_rule == 1;
    const int wstride = gridDim.x * (blockDim.x >> 5);
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += wstride) {
        const int z = row / a.ny, y = row - z * a.ny;
        if (y < 1 || y > a.ny - 2 || (RANK == 3 && (z < 1 || z > a.nz - 2))) continue;  // warp-uniform
        const int8_t* sr = a.s + (int64_t)row * a.nx;
        const uint8_t* er = eqm + (int64_t)row * a.nx;
        uint32_t carry = 0;  // S word of the previous step (its byte 3 is the left neighbour)
        for (int x0s = 0; x0s < a.nx; x0s += 128) {
            const int x0 = x0s + 4 * lane;
            const uint32_t cw = load4_s8(sr, x0, a.nx, vec);
            uint32_t xmw = __shfl_up_sync(kFull, cw, 1);
            uint32_t xpw = __shfl_down_sync(kFull, cw, 1);
            const uint32_t last = __shfl_sync(kFull, cw, 31);
            if (lane == 0) xmw = carry;
            if (lane == 31) xpw = x0 + 4 < a.nx ? (uint32_t)(uint8_t)__ldg(sr + x0 + 4) : 0u;
            carry = last;
            const uint32_t eqw = literal ? 0xFFFFFFFFu : load4_s8(reinterpret_cast<const int8_t*>(er), x0, a.nx, vec);
            // byte k of sel(bit) = 0xFF if bit `bit` of equal-q mask byte k is set
            auto sel = [&](int bit) -> uint32_t { return __vcmpne4(eqw & (0x01010101u << bit), 0u); };
            uint32_t b2 = (__vcmpne4(__byte_perm(xmw, cw, 0x6543), cw) & sel(4)) |
                          (__vcmpne4(__byte_perm(cw, xpw, 0x4321), cw) & sel(5)) |
                          (__vcmpne4(load4_s8(sr - a.nx, x0, a.nx, vec), cw) & sel(2)) |
                          (__vcmpne4(load4_s8(sr + a.nx, x0, a.nx, vec), cw) & sel(3));
            if (RANK == 3) {
                b2 |= (__vcmpne4(load4_s8(sr - plane, x0, a.nx, vec), cw) & sel(0)) |
                      (__vcmpne4(load4_s8(sr + plane, x0, a.nx, vec), cw) & sel(1));
            }
            unsigned nib = ((b2 & 0x80808080u) * 0x00204081u) >> 28;
#pragma unroll
            for (int j = 0; j < 4; ++j)  // interior along x; bytes past the row end are not points
                if (x0 + j < 1 || x0 + j > a.nx - 2) nib &= ~(1u << j);
            append_sites(a, sb, nib, x0, y, z);
        }
    }
}

// Exact Dist2 of each query left by k_query: min over the listed B2 sites.
// CTA i takes 256 queries (block i % qb) against one slice of the site list
// (i / qb), staged through shared memory; each thread folds its minimum into
// fmin with an atomic, and the last CTA to finish writes the outputs.
constexpr int kBruteChunk = 1024;
__global__ void __launch_bounds__(256) k_brute(RouteArgs a)
{
    wait_prior_grid();
    volatile int* ctr = a.ctr;
    if (ctr[kCtrDense] || ctr[kCtrUnresolved] == 0) return;
    const int nf = ctr[kCtrFailed];
    const int nb = ctr[kCtrB2];
    const int qblocks = (nf + blockDim.x - 1) / blockDim.x;
    if (nf > a.fcap || nb > a.b2cap || (long long)nf * nb > a.brute_budget || qblocks > (int)gridDim.x) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr[kCtrDense] = 1;
        return;
    }
    __shared__ uint2 sites[kBruteChunk];
    __shared__ int last;
    const uint2* list = reinterpret_cast<const uint2*>(a.b2list);
    const int plane = a.ny * a.nx;
    const int qb = qblocks;
    const int slices = max(1, (int)gridDim.x / qb);
    const int qblk = blockIdx.x % qb, slice = blockIdx.x / qb;
    if (slice < slices) {
        const int per = (nb + slices - 1) / slices;
        const int b0 = min(nb, slice * per), b1 = min(nb, b0 + per);
        const int f = qblk * blockDim.x + threadIdx.x;
        int x = 0, y = 0, z = 0;
        if (f < nf) {
            const int idx = a.flist[f].idx;
            z = idx / plane;
            const int rem = idx - z * plane;
            y = rem / a.nx;
            x = rem - y * a.nx;
        }
        int best = kDistInf;
        for (int c0 = b0; c0 < b1; c0 += kBruteChunk) {
            const int n = min(kBruteChunk, b1 - c0);
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) sites[i] = list[c0 + i];
            __syncthreads();
            for (int i = 0; i < n; ++i) {
                const uint2 b = sites[i];
                const int dx = (int)(b.x & 0xFFFFu) - x, dy = (int)(b.x >> 16) - y, dz = (int)b.y - z;
                best = min(best, dz * dz + dy * dy + dx * dx);
            }
        }
        if (f < nf && best < kDistInf) atomicMin(a.fmin + f, best);  // -1 (done) stays
    }
    // the last CTA writes every output (no B2 at all: Dist2 = INF, w = 1)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(a.ctr + kCtrBruteDone, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        for (int f = threadIdx.x; f < nf; f += blockDim.x) {
            const int32_t d2 = *static_cast<volatile int32_t*>(a.fmin + f);
            if (d2 < 0) continue;  // the second shell search found it
            const Query e = a.flist[f];
            emit_query(a, e, d2);
        }
    }
}

}  // namespace

int route_table_r2(int rank) { return rank == 2 ? kTableR2_2 : kTableR2; }

cudaError_t launch_route_query(const RouteArgs& a, int blocks, cudaStream_t st)
{
    return a.rank == 3 ? launch_chained(k_query<3>, dim3(blocks), dim3(256), 0, st, a)
                       : launch_chained(k_query<2>, dim3(blocks), dim3(256), 0, st, a);
}

cudaError_t launch_route_query_mid(const RouteArgs& a, int blocks, cudaStream_t st)
{
    return a.rank == 3 ? launch_chained(k_query_mid<3>, dim3(blocks), dim3(256), 0, st, a)
                       : launch_chained(k_query_mid<2>, dim3(blocks), dim3(256), 0, st, a);
}

cudaError_t launch_route_query_far(const RouteArgs& a, int blocks, cudaStream_t st)
{
    return a.rank == 3 ? launch_chained(k_query_far<3>, dim3(blocks), dim3(256), 0, st, a)
                       : launch_chained(k_query_far<2>, dim3(blocks), dim3(256), 0, st, a);
}

cudaError_t launch_route_b2sites(const RouteArgs& a, int blocks, cudaStream_t st)
{
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; };
    const int vec = (a.nx % 4 == 0) && al(a.s) && al(a.eqm);
    return a.rank == 3 ? launch_chained(k_b2sites<3>, dim3(blocks), dim3(256), 0, st, a, vec)
                       : launch_chained(k_b2sites<2>, dim3(blocks), dim3(256), 0, st, a, vec);
}

cudaError_t launch_route_brute(const RouteArgs& a, int blocks, cudaStream_t st)
{
    return launch_chained(k_brute, dim3(blocks), dim3(256), 0, st, a);
}

}  // namespace qai
