// qai_signed.cu -- the signed-point route of the second EDT (step D) and of
// step E.
//
// Step E adds C = S w eta eps (Sec. VI-E). Where S = 0 the output is D'
// whatever Dist2 is, and on B1 (Dist1 = 0) the weight is 1 whatever Dist2 is
// (the boundary value eta eps); the step-A kernel writes both of these
// outputs. Dist2 is needed only at the queries -- points with S != 0 off
// B1 -- which the first EDT lists with their Dist1 and sign. These kernels
// give the exact Dist2 of every query, Eq. 2 over the sign-flipping boundary
// B2 of Algorithm 3:
//
// Two routes. The sparse one, where the signed points (S != 0) are few enough
// to be listed: k_b2sparse lists the B2 sites from the signed set and
// k_brute (sparse) gives every query the minimum over them. The bitmap route,
// where they are not or the product of queries and sites is over its budget:
//
//   k_b2map    GetBoundary(S) at every interior point, bit-parallel from the
//              packed S map and the differ maps of step A: the B2 bitmap, 1
//              bit a point.
//   k_query    one thread per query: the 3 x 3 x 3 block of the bitmap around
//              it (every point within squared distance 3, and no other).
//   k_query_mid one warp per query the first left: the bitmap rows within
//              radius R (12 in 3-D, 31 in 2-D) of it, each row's nearest bit
//              to x by bit scans; the minimum is exact when it is <= R^2.
//   k_b2list   (only when queries remain) lists the B2 sites from the bitmap;
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

// Radius of the second shell phase (in grid units), 3-D and 2-D. The 3-D
// phase reads the bitmap rows (dz, dy) with dz^2 + dy^2 <= R^2; the window
// of a row is 2R + 1 <= 63 bits.
constexpr int kMidR3 = 12, kMidR2 = 31;
constexpr int count_rows3(int r)
{
    int n = 0;
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            if (dz * dz + dy * dy <= r * r) ++n;
    return n;
}
constexpr int kRows3 = count_rows3(kMidR3);
struct RowTable3 {
    int8_t dz[kRows3], dy[kRows3];
};
constexpr RowTable3 make_rows3()
{
    RowTable3 t{};
    int n = 0;
    for (int dz = -kMidR3; dz <= kMidR3; ++dz)
        for (int dy = -kMidR3; dy <= kMidR3; ++dy)
            if (dz * dz + dy * dy <= kMidR3 * kMidR3) {
                t.dz[n] = (int8_t)dz;
                t.dy[n] = (int8_t)dy;
                ++n;
            }
    return t;
}
static_assert(2 * kMidR3 + 1 <= 63 && 2 * kMidR2 + 1 <= 63, "shell windows fit 64 bits");
__constant__ RowTable3 c_rows3 = make_rows3();

constexpr int kMidBuf = 2048;  // per-CTA buffer of the first phase's leftovers

// The low bit of every nonzero 2-bit field of v.
__device__ __forceinline__ uint32_t field_lsb(uint32_t v) { return (v | (v >> 1)) & 0x55555555u; }

// Bits 0, 2, 4, ..., 30 of v to bits 0..15.
__device__ __forceinline__ uint32_t even_bits(uint32_t v)
{
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0F0F0F0Fu;
    v = (v | (v >> 4)) & 0x00FF00FFu;
    return (v | (v >> 8)) & 0x0000FFFFu;
}

__device__ __forceinline__ void coords(const RouteArgs& a, int idx, int& x, int& y, int& z)
{
    const int plane = a.ny * a.nx;
    z = idx / plane;
    const int rem = idx - z * plane;
    y = rem / a.nx;
    x = rem - y * a.nx;
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

// Packed word k of row `prow` (0 past the row).
__device__ __forceinline__ uint32_t sword(const RouteArgs& a, int64_t prow, int k, bool ok)
{
    return ok && k >= 0 && k < a.wpr ? __ldg(a.spk + prow * a.wpr + k) : 0u;
}

// Packed word k of map m, row `prow` (0 past the row, or where ok is false).
__device__ __forceinline__ uint32_t mword(const uint32_t* m, int64_t prow, int k, int wpr, bool ok)
{
    return ok && k >= 0 && k < wpr ? __ldg(m + prow * wpr + k) : 0u;
}

// Rows of a plane a warp takes at once in the B2 map.
constexpr int kMapRows = 4;

// The B2 bitmap: GetBoundary(S) (Algorithm 3) at every interior point, 16
// points (one packed S word) per lane, bit-parallel: a point is on B2 when an
// axis neighbour has a different S and (the default rule) the same q, which
// the differ maps of step A give (the -x, -y, -z pairs through the
// neighbour's +x, +y, +z bit). A warp takes kMapRows rows of a plane with all
// their words loaded up front; pairs of lanes make one bitmap word. Every
// word is written (the bitmap is not cleared between calls). Nothing to do
// without queries.
template <int RANK>
__device__ __forceinline__ void k_b2map_body(const RouteArgs& a, const int bx, const int gx)
{
    wait_prior_grid();
    const volatile int* ctr = a.ctr;
    if (ctr[kCtrDense] || !ctr[kCtrBitmap]) return;
    const int lane = threadIdx.x & 31;
    const int wpr = a.wpr;
    const bool literal = a.m.b2_rule == 1;
    const int yb = (a.ny + kMapRows - 1) / kMapRows;
    const int items = a.nz * yb;
    const int wstride = gx * (blockDim.x >> 5);
    constexpr uint32_t kLo = 0x55555555u;
    for (int it = bx * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items; it += wstride) {
        const int z = RANK == 3 ? it / yb : 0;
        const int y0 = (it - z * yb) * kMapRows;
        const int64_t row0 = (int64_t)z * a.ny + y0;
        for (int ks = 0; ks < wpr; ks += 32) {
            const int k = ks + lane;
            // S of rows y0 - 1 .. y0 + kMapRows and of planes z -+ 1; the
            // differ words of rows y0 - 1 .. y0 + kMapRows - 1 and of plane
            // z - 1
            uint32_t sy[kMapRows + 2], szm[kMapRows], szp[kMapRows], ey[kMapRows + 1], ez[kMapRows], ezm[kMapRows];
            uint32_t any = 0;
#pragma unroll
            for (int i = 0; i < kMapRows + 2; ++i) {
                const int y = y0 - 1 + i;
                sy[i] = mword(a.spk, row0 - 1 + i, k, wpr, y >= 0 && y < a.ny);
                any |= sy[i];
            }
#pragma unroll
            for (int i = 0; i < kMapRows; ++i) {
                const bool ok = RANK == 3 && y0 + i < a.ny;
                szm[i] = mword(a.spk, row0 + i - a.ny, k, wpr, ok && z > 0);
                szp[i] = mword(a.spk, row0 + i + a.ny, k, wpr, ok && z < a.nz - 1);
                any |= szm[i] | szp[i];
            }
            if (!__any_sync(kFull, any != 0)) {
                // S = 0 around every point of these rows: no B2 point
#pragma unroll
                for (int i = 0; i < kMapRows; ++i)
                    if (y0 + i < a.ny && !(lane & 1) && k < wpr) a.b2bits[(row0 + i) * a.bwpr + (k >> 1)] = 0u;
                continue;
            }
            if (!literal) {
#pragma unroll
                for (int i = 0; i <= kMapRows; ++i) {
                    const int y = y0 - 1 + i;
                    ey[i] = mword(a.nexy, row0 - 1 + i, k, wpr, y >= 0 && y < a.ny);
                }
#pragma unroll
                for (int i = 0; i < kMapRows; ++i) {
                    const bool ok = RANK == 3 && y0 + i < a.ny;
                    ez[i] = mword(a.nez, row0 + i, k, wpr, ok);
                    ezm[i] = mword(a.nez, row0 + i - a.ny, k, wpr, ok && z > 0);
                }
            }
            // interior along x: fields 16k + i in [1, nx - 2]
            uint32_t inner = k < wpr ? 0xFFFFFFFFu : 0u;
            if (k == 0) inner &= ~3u;
            const int last = a.nx - 2 - 16 * k;  // last inner field
            if (last < 15) inner &= last < 0 ? 0u : (1u << (2 * (last + 1))) - 1u;
#pragma unroll
            for (int i = 0; i < kMapRows; ++i) {
                const int y = y0 + i;
                if (y >= a.ny) break;  // warp-uniform
                const uint32_t w = sy[i + 1];
                uint32_t wl = __shfl_up_sync(kFull, w, 1), wr = __shfl_down_sync(kFull, w, 1);
                if (lane == 0) wl = mword(a.spk, row0 + i, k - 1, wpr, true);
                if (lane == 31) wr = mword(a.spk, row0 + i, k + 1, wpr, true);
                uint32_t exl = 0;
                if (!literal) {
                    exl = __shfl_up_sync(kFull, ey[i + 1], 1);
                    if (lane == 0) exl = mword(a.nexy, row0 + i, k - 1, wpr, true);
                }
                const bool row_inner = y >= 1 && y <= a.ny - 2 && (RANK == 2 || (z >= 1 && z <= a.nz - 2));
                // differing neighbours, per direction
                const uint32_t dxm = field_lsb(__funnelshift_l(wl, w, 2) ^ w);
                const uint32_t dxp = field_lsb(__funnelshift_r(w, wr, 2) ^ w);
                const uint32_t dym = field_lsb(sy[i] ^ w), dyp = field_lsb(sy[i + 2] ^ w);
                const uint32_t dzm = RANK == 3 ? field_lsb(szm[i] ^ w) : 0u;
                const uint32_t dzp = RANK == 3 ? field_lsb(szp[i] ^ w) : 0u;
                uint32_t b2;
                if (literal) {
                    b2 = dxm | dxp | dym | dyp | dzm | dzp;
                } else {
                    // a pair counts where its differ bit is clear (the same q)
                    const uint32_t nxy = ey[i + 1];
                    b2 = (dxp & ~nxy) | (dxm & ~__funnelshift_l(exl, nxy, 2)) | (dyp & ~(nxy >> 1)) |
                         (dym & ~(ey[i] >> 1));
                    if (RANK == 3) b2 |= (dzp & ~ez[i]) | (dzm & ~ezm[i]);
                    b2 &= kLo;
                }
                b2 = row_inner ? b2 & inner : 0u;
                const uint32_t m16 = even_bits(b2);
                const uint32_t hi = __shfl_down_sync(kFull, m16, 1);
                if (!(lane & 1) && k < wpr) a.b2bits[(row0 + i) * a.bwpr + (k >> 1)] = m16 | (hi << 16);
            }
        }
    }
}

template <int RANK>
__global__ void __launch_bounds__(256, 3) k_b2map(RouteArgs a)
{
    k_b2map_body<RANK>(a, blockIdx.x, gridDim.x);
}


// Bitmap bits x0 .. x0 + 63 of row `prow` (0 outside the row).
__device__ __forceinline__ uint64_t bwin64(const RouteArgs& a, int64_t prow, int x0)
{
    const int lo = x0 >> 5, sh = x0 & 31;  // arithmetic shift: lo = -1 or -2 left of the row
    const uint32_t* r = a.b2bits + prow * a.bwpr;
    auto w = [&](int i) { return i >= 0 && i < a.bwpr ? __ldg(r + i) : 0u; };
    const uint32_t w0 = w(lo), w1 = w(lo + 1), w2 = w(lo + 2);
    return (uint64_t)__funnelshift_r(w0, w1, sh) | ((uint64_t)__funnelshift_r(w1, w2, sh) << 32);
}

// Squared distance from bit R of v to its nearest set bit among bits 0..2R
// (INT_MAX if none).
__device__ __forceinline__ int nearest_bit2(uint64_t v, int R)
{
    const uint64_t left = v & ((2ull << R) - 1ull);   // bits 0..R
    const uint64_t right = (v >> R) & ((2ull << R) - 1ull);  // bits R..2R, from R
    int d = 0x7FFFFFFF;
    if (left) {
        const int hb = 63 - __clzll((long long)left);
        d = min(d, R - hb);
    }
    if (right) d = min(d, __ffsll((long long)right) - 1);
    return d == 0x7FFFFFFF ? d : d * d;
}

// Leftover of a shell phase to the next one (per-CTA buffer, one atomic).
struct LeftBuf {
    Query* e;
    int* n;
};

template <int RANK>
__device__ __forceinline__ void k_query_body(const RouteArgs& a, const int bx, const int gx)
{
    wait_prior_grid();
    volatile int* ctr = a.ctr;
    if (ctr[kCtrDense] || !ctr[kCtrBitmap]) return;
    const int nq = ctr[kCtrQueries];
    __shared__ Query mbuf[kMidBuf];
    __shared__ int mn, mbase;
    if (threadIdx.x == 0) mn = 0;
    __syncthreads();
    for (int i = bx * blockDim.x + threadIdx.x; i < nq; i += gx * blockDim.x) {
        const Query e = a.qlist[i];
        int found = 0x7FFFFFFF;
        if (a.shell) {
            int x, y, z;
            coords(a, e.idx, x, y, z);
            const int64_t row = (int64_t)z * a.ny + y;
#pragma unroll
            for (int dz = (RANK == 3 ? -1 : 0); dz <= (RANK == 3 ? 1 : 0); ++dz)
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy) {
                    if ((unsigned)(y + dy) >= (unsigned)a.ny || (RANK == 3 && (unsigned)(z + dz) >= (unsigned)a.nz))
                        continue;
                    const uint32_t v = (uint32_t)bwin64(a, row + (int64_t)dz * a.ny + dy, x - 1) & 7u;
                    const int d = nearest_bit2(v, 1);
                    if (d != 0x7FFFFFFF) found = min(found, dz * dz + dy * dy + d);
                }
        }
        if (found <= 3) {  // every point within squared distance 3 is in the block
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

template <int RANK>
__global__ void __launch_bounds__(256) k_query(RouteArgs a)
{
    k_query_body<RANK>(a, blockIdx.x, gridDim.x);
}


// Second phase: one warp per query; the lanes take the bitmap rows within
// radius R, each row's nearest bit to x in the window x - R .. x + R.
template <int RANK>
__device__ __forceinline__ void k_query_mid_body(const RouteArgs& a, const int bx, const int gx)
{
    wait_prior_grid();
    volatile int* ctr = a.ctr;
    if (ctr[kCtrDense] || !ctr[kCtrBitmap]) return;
    const int nm = min((int)ctr[kCtrMid], a.qcap);
    const int lane = threadIdx.x & 31;
    const int wstride = gx * (blockDim.x >> 5);
    constexpr int R = RANK == 3 ? kMidR3 : kMidR2;
    constexpr int nrows = RANK == 3 ? kRows3 : 2 * kMidR2 + 1;
    for (int i = bx * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nm; i += wstride) {
        const Query e = a.mlist[i];
        int best = 0x7FFFFFFF;
        if (a.shell) {
            int x, y, z;
            coords(a, e.idx, x, y, z);
            const int64_t row = (int64_t)z * a.ny + y;
            for (int r = lane; r < nrows; r += 32) {
                const int dz = RANK == 3 ? c_rows3.dz[r] : 0;
                const int dy = RANK == 3 ? c_rows3.dy[r] : r - kMidR2;
                if ((unsigned)(y + dy) >= (unsigned)a.ny || (RANK == 3 && (unsigned)(z + dz) >= (unsigned)a.nz))
                    continue;
                const int d = nearest_bit2(bwin64(a, row + (int64_t)dz * a.ny + dy, x - R), R);
                if (d != 0x7FFFFFFF) best = min(best, dz * dz + dy * dy + d);
            }
            best = __reduce_min_sync(kFull, best);
        }
        if (lane == 0) {
            if (best <= R * R) {  // exact: a nearer site would lie in a row and window read here
                emit_query(a, e, best);
            } else {
                const int k = atomicAdd(a.ctr + kCtrUnresolved, 1);
                if (k < a.fcap) {
                    a.flist[k] = e;
                    a.fmin[k] = kDistInf;
                }
            }
        }
    }
}

template <int RANK>
__global__ void __launch_bounds__(256) k_query_mid(RouteArgs a)
{
    k_query_mid_body<RANK>(a, blockIdx.x, gridDim.x);
}


// The B2 sites, listed from the bitmap (only when some query is left to
// the search over them): one thread per bitmap word, warp-aggregated appends
// into a per-CTA buffer, one global atomic per CTA.
constexpr int kSiteBuf = 2048;
__device__ __forceinline__ void k_b2list_body(const RouteArgs& a, const int bx, const int gx)
{
    wait_prior_grid();
    volatile int* ctr = a.ctr;
    if (ctr[kCtrDense] || !ctr[kCtrBitmap] || ctr[kCtrUnresolved] == 0) return;
    __shared__ uint2 sbuf[kSiteBuf];
    __shared__ int sn, sfull, sbase;  // sfull: first reservation that did not fit
    if (threadIdx.x == 0) {
        sn = 0;
        sfull = kSiteBuf;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t words = (int64_t)a.nz * a.ny * a.bwpr;
    const int64_t stride = (int64_t)gx * blockDim.x;
    uint2* glist = reinterpret_cast<uint2*>(a.b2list);
    for (int64_t base = (int64_t)bx * blockDim.x; base < words; base += stride) {
        const int64_t i = base + threadIdx.x;
        uint32_t w = i < words ? __ldg(a.b2bits + i) : 0u;
        const int cnt = __popc(w);
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += v;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        if (total == 0) continue;
        int wbase = 0;
        if (lane == 31) wbase = atomicAdd(&sn, total);
        wbase = __shfl_sync(kFull, wbase, 31);
        const bool global = wbase + total > kSiteBuf;
        if (global && lane == 31) {
            atomicMin(&sfull, wbase);  // every later reservation fails too (sn only grows)
            wbase = atomicAdd(a.ctr + kCtrB2, total);
        }
        if (global) wbase = __shfl_sync(kFull, wbase, 31);
        uint2* list = global ? glist : sbuf;
        const int cap = global ? a.b2cap : kSiteBuf;
        int pos = wbase + incl - cnt;
        if (w) {
            const int64_t row = i / a.bwpr;
            const int x0 = 32 * (int)(i - row * a.bwpr);
            const int z = (int)(row / a.ny), y = (int)(row - (int64_t)z * a.ny);
            for (; w; w &= w - 1, ++pos)
                if (pos < cap) list[pos] = make_uint2((uint32_t)(x0 + __ffs(w) - 1) | ((uint32_t)y << 16), (uint32_t)z);
        }
    }
    __syncthreads();
    const int n = min(sn, sfull);
    if (threadIdx.x == 0) sbase = n > 0 ? atomicAdd(a.ctr + kCtrB2, n) : 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n && sbase + i < a.b2cap; i += blockDim.x) glist[sbase + i] = sbuf[i];
}

__global__ void __launch_bounds__(256) k_b2list(RouteArgs a)
{
    k_b2list_body(a, blockIdx.x, gridDim.x);
}


// S code (0, 1: +1, 2: -1) of point (x, y, z) from the packed S map; 0
// outside the field.
__device__ __forceinline__ int s_at(const RouteArgs& a, int x, int y, int z)
{
    if ((unsigned)x >= (unsigned)a.nx || (unsigned)y >= (unsigned)a.ny || (unsigned)z >= (unsigned)a.nz) return 0;
    const uint32_t w = __ldg(a.spk + ((int64_t)z * a.ny + y) * a.wpr + (x >> 4));
    return (int)((w >> (2 * (x & 15))) & 3u);
}

// Whether q differs across the pair (x, y, z) -- (x, y, z) + e, e the unit
// step along axis 0 (z), 1 (y) or 2 (x): the differ bit of the pair's lower
// point (both points inside the field).
__device__ __forceinline__ bool q_differs(const RouteArgs& a, int x, int y, int z, int axis)
{
    const int64_t w = ((int64_t)z * a.ny + y) * a.wpr + (x >> 4);
    const int sh = 2 * (x & 15);
    if (axis == 0) return (__ldg(a.nez + w) >> sh) & 1u;
    return (__ldg(a.nexy + w) >> (sh + (axis == 1 ? 1 : 0))) & 1u;
}

// GetBoundary(S) (Algorithm 3) at the interior point (x, y, z) with S code sc:
// an axis neighbour with a different S and (the default rule) the same q.
template <int RANK>
__device__ __forceinline__ bool is_b2(const RouteArgs& a, int x, int y, int z, int sc)
{
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int axis = k >> 1;
        if (RANK == 2 && axis == 0) continue;
        const int sg = (k & 1) ? 1 : -1;
        const int nx_ = x + (axis == 2 ? sg : 0), ny_ = y + (axis == 1 ? sg : 0), nz_ = z + (axis == 0 ? sg : 0);
        if (s_at(a, nx_, ny_, nz_) == sc) continue;
        if (a.m.b2_rule == 1) return true;
        // the pair's lower point carries its differ bit
        if (!(sg > 0 ? q_differs(a, x, y, z, axis) : q_differs(a, nx_, ny_, nz_, axis))) return true;
    }
    return false;
}

// The B2 sites from the signed set -- the listed B1 points with S != 0 and the
// queries (S != 0 off B1): GetBoundary(S) compares S across a pair, so every
// B2 site is a signed point or an axis neighbour of one. Each signed point p
// has a thread for itself and one for each axis neighbour with S = 0; such a
// neighbour is tested only by its signed neighbour of smallest linear index,
// so no site is listed twice. The sites go to the site list (warp-aggregated
// appends into a per-CTA buffer, one global atomic per CTA); fmin of every
// query starts at INF. A signed list that overflowed hands the field to the
// bitmap route.
constexpr int kSparseBuf = 2048;
template <int RANK>
__device__ __forceinline__ void k_b2sparse_body(const RouteArgs& a, const int bx, const int gx)
{
    wait_prior_grid();
    volatile int* ctr = a.ctr;
    if (ctr[kCtrDense]) return;
    const int nq = ctr[kCtrQueries];
    if (nq > a.qcap) {  // the query list is incomplete: the dense route takes over
        if (bx == 0 && threadIdx.x == 0) ctr[kCtrDense] = 1;
        return;
    }
    if (nq == 0) return;  // no point needs Dist2
    const int ns = ctr[kCtrSigned];
    if (ctr[kCtrSignedOver] || ns > a.scap || !a.shell || nq > a.fcap) {
        if (bx == 0 && threadIdx.x == 0) ctr[kCtrBitmap] = 1;
        return;
    }
    if (bx == 0 && threadIdx.x == 0) ctr[kCtrUnresolved] = nq;  // every query takes the site search
    for (int i = bx * blockDim.x + threadIdx.x; i < nq; i += gx * blockDim.x) a.fmin[i] = kDistInf;
    __shared__ uint2 sbuf[kSparseBuf];
    __shared__ int sn, sfull, sbase;
    if (threadIdx.x == 0) {
        sn = 0;
        sfull = kSparseBuf;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int plane = a.ny * a.nx;
    uint2* glist = reinterpret_cast<uint2*>(a.b2list);
    const int items = ns + nq;
    // eight threads per signed point, one per candidate: c = 0 the point
    // itself, c = 1 .. 6 its axis neighbours z-, z+, y-, y+, x-, x+ (c = 7
    // idle), so that the chains of dependent loads run side by side
    const int64_t slots = (int64_t)items * 8;
    for (int64_t base = (int64_t)bx * blockDim.x; base < slots; base += (int64_t)gx * blockDim.x) {
        const int64_t slot = base + threadIdx.x;
        const int item = (int)(slot >> 3), c = (int)(slot & 7);
        uint2 found[1];
        int nfound = 0;
        const bool live = slot < slots && c <= 6 && !(RANK == 2 && (c == 1 || c == 2));
        if (live) {
            const int p = item < ns ? a.slist[item] : a.qlist[item - ns].idx;
            const int z = p / plane, rem = p - z * plane;
            const int y = rem / a.nx, x = rem - y * a.nx;
            int cz = 0, cy = 0, cx = 0;
            if (c > 0) {
                const int axis = (c - 1) >> 1;
                const int sg = (c - 1) & 1 ? 1 : -1;
                (axis == 0 ? cz : (axis == 1 ? cy : cx)) = sg;
            }
            const int bx_ = x + cx, by = y + cy, bz = z + cz;
            const bool inner = (unsigned)(bx_ - 1) < (unsigned)(a.nx - 2) &&
                               (unsigned)(by - 1) < (unsigned)(a.ny - 2) &&
                               (RANK == 2 || (unsigned)(bz - 1) < (unsigned)(a.nz - 2));
            if (inner) {
                const int sc = s_at(a, bx_, by, bz);
                bool test = true;
                if (c > 0) {
                    // a signed point lists itself; an S = 0 neighbour is
                    // owned by p when no signed neighbour of it precedes p:
                    // an offset (from p) precedes 0 in (dz, dy, dx) order
                    // exactly when its point precedes p
                    test = sc == 0;
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        const int axis = k >> 1;
                        if (RANK == 2 && axis == 0) continue;
                        const int sg = (k & 1) ? 1 : -1;
                        const int oz = cz + (axis == 0 ? sg : 0), oy = cy + (axis == 1 ? sg : 0),
                                  ox = cx + (axis == 2 ? sg : 0);
                        const bool before = oz < 0 || (oz == 0 && (oy < 0 || (oy == 0 && ox < 0)));
                        if (test && before && s_at(a, x + ox, y + oy, z + oz) != 0) test = false;
                    }
                }
                if (test && is_b2<RANK>(a, bx_, by, bz, sc))
                    found[nfound++] = make_uint2((uint32_t)bx_ | ((uint32_t)by << 16), (uint32_t)bz);
            }
        }
        // warp-aggregated append of the found sites
        int incl = nfound;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += v;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        if (total == 0) continue;
        int wbase = 0;
        if (lane == 31) wbase = atomicAdd(&sn, total);
        wbase = __shfl_sync(kFull, wbase, 31);
        const bool global = wbase + total > kSparseBuf;
        if (global && lane == 31) {
            atomicMin(&sfull, wbase);  // every later reservation fails too (sn only grows)
            wbase = atomicAdd(a.ctr + kCtrB2, total);
        }
        if (global) wbase = __shfl_sync(kFull, wbase, 31);
        uint2* list = global ? glist : sbuf;
        const int cap = global ? a.b2cap : kSparseBuf;
        int pos = wbase + incl - nfound;
        for (int f = 0; f < nfound; ++f, ++pos)
            if (pos < cap) list[pos] = found[f];
    }
    __syncthreads();
    const int n = min(sn, sfull);
    if (threadIdx.x == 0) sbase = n > 0 ? atomicAdd(a.ctr + kCtrB2, n) : 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n && sbase + i < a.b2cap; i += blockDim.x) glist[sbase + i] = sbuf[i];
}

template <int RANK>
__global__ void __launch_bounds__(256) k_b2sparse(RouteArgs a)
{
    k_b2sparse_body<RANK>(a, blockIdx.x, gridDim.x);
}


// Exact Dist2 of queries by a search over every listed B2 site: all queries
// (sparse: the sparse route) or those the shell phases left (the bitmap
// route). CTA i takes 256 queries (block i % qb) against one slice of the
// site list (i / qb), staged through shared memory; each thread folds its
// minimum into fmin with an atomic, and the last CTA to finish writes the
// outputs. Over the budget, the sparse route hands over to the bitmap route
// and the bitmap route to the dense second EDT.
constexpr int kBruteChunk = 1024;
__device__ __forceinline__ void k_brute_body(const RouteArgs& a, int sparse, const int bx, const int gx)
{
    wait_prior_grid();
    volatile int* ctr = a.ctr;
    if (ctr[kCtrDense]) return;
    if (sparse ? (ctr[kCtrBitmap] || ctr[kCtrQueries] == 0) : (!ctr[kCtrBitmap] || ctr[kCtrUnresolved] == 0))
        return;
    const int nf = sparse ? ctr[kCtrQueries] : ctr[kCtrUnresolved];
    const int nb = ctr[kCtrB2];
    const int qblocks = (nf + blockDim.x - 1) / blockDim.x;
    if (nf > a.fcap || nb > a.b2cap || (long long)nf * nb > a.brute_budget || qblocks > (int)gx) {
        if (bx == 0 && threadIdx.x == 0) {
            if (sparse) {  // the bitmap route starts its own counts
                ctr[kCtrUnresolved] = 0;
                ctr[kCtrB2] = 0;
                ctr[kCtrBitmap] = 1;
            } else {
                ctr[kCtrDense] = 1;
            }
        }
        return;
    }
    const Query* src = sparse ? a.qlist : a.flist;
    __shared__ uint2 sites[kBruteChunk];
    __shared__ int last;
    const uint2* list = reinterpret_cast<const uint2*>(a.b2list);
    const int plane = a.ny * a.nx;
    const int qb = qblocks;
    const int slices = max(1, (int)gx / qb);
    const int qblk = bx % qb, slice = bx / qb;
    if (slice < slices) {
        const int per = (nb + slices - 1) / slices;
        const int b0 = min(nb, slice * per), b1 = min(nb, b0 + per);
        const int f = qblk * blockDim.x + threadIdx.x;
        int x = 0, y = 0, z = 0;
        if (f < nf) {
            const int idx = src[f].idx;
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
        if (f < nf && best < kDistInf) atomicMin(a.fmin + f, best);
    }
    // the last CTA writes every output (no B2 at all: Dist2 = INF, w = 1)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(a.ctr + kCtrBruteDone, 1) == (int)gx - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        for (int f = threadIdx.x; f < nf; f += blockDim.x) {
            const int32_t d2 = *static_cast<volatile int32_t*>(a.fmin + f);
            emit_query(a, src[f], d2);
        }
    }
}

__global__ void __launch_bounds__(256) k_brute(RouteArgs a, int sparse)
{
    k_brute_body(a, sparse, blockIdx.x, gridDim.x);
}


// A grid-stride kernel's grid: every CTA resident at once.
template <class K>
int resident(K kern)
{
    int dev = 0, sms = 152, per = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0) != cudaSuccess || per < 1) per = 1;
    return sms * per;
}

}  // namespace

cudaError_t launch_route_b2map(const RouteArgs& a, cudaStream_t st)
{
    auto run = [&](auto kern) { return launch_chained(kern, dim3(resident(kern)), dim3(256), 0, st, a); };
    return a.rank == 3 ? run(k_b2map<3>) : run(k_b2map<2>);
}

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

cudaError_t launch_route_b2list(const RouteArgs& a, cudaStream_t st)
{
    return launch_chained(k_b2list, dim3(resident(k_b2list)), dim3(256), 0, st, a);
}

cudaError_t launch_route_brute(const RouteArgs& a, int blocks, bool sparse, cudaStream_t st)
{
    return launch_chained(k_brute, dim3(blocks), dim3(256), 0, st, a, sparse ? 1 : 0);
}

namespace {
// Grouped kernels over fields of either rank: the body instance is picked
// per work item from the field's arguments.
#define QAI_ROUTE_GROUP(NAME, LB)                                                   \
    __global__ void __launch_bounds__(LB) NAME##_group(const __grid_constant__ GroupQueue q) \
    {                                                                               \
        run_group<RouteArgs>(q, [&](const RouteArgs& a, int b, int n) {             \
            if (a.rank == 3) NAME##_body<3>(a, b, n);                               \
            else NAME##_body<2>(a, b, n);                                           \
        });                                                                         \
    }
QAI_ROUTE_GROUP(k_b2map, 256)
QAI_ROUTE_GROUP(k_query, 256)
QAI_ROUTE_GROUP(k_query_mid, 256)
QAI_ROUTE_GROUP(k_b2sparse, 256)
#undef QAI_ROUTE_GROUP

__global__ void __launch_bounds__(256) k_b2list_group(const __grid_constant__ GroupQueue q)
{
    run_group<RouteArgs>(q, [&](const RouteArgs& a, int b, int n) { k_b2list_body(a, b, n); });
}

__global__ void __launch_bounds__(256) k_brute_group(const __grid_constant__ GroupQueue q, int sparse)
{
    run_group<RouteArgs>(q, [&](const RouteArgs& a, int b, int n) { k_brute_body(a, sparse, b, n); });
}

template <class K, class... A>
cudaError_t run_grouped(K kern, const GroupQueue& q, cudaStream_t st, A... extra)
{
    const int grid = std::min(group_total(q), persistent_grid(kern, 256, 0));
    if (grid < 1) return cudaSuccess;
    return launch_chained(kern, dim3(grid), dim3(256), 0, st, q, extra...);
}
}  // namespace

cudaError_t launch_group_route(RouteKernel k, const GroupQueue& q, cudaStream_t st)
{
    switch (k) {
    case kRouteB2Sparse: return run_grouped(k_b2sparse_group, q, st);
    case kRouteBruteSparse: return run_grouped(k_brute_group, q, st, 1);
    case kRouteB2Map: return run_grouped(k_b2map_group, q, st);
    case kRouteQuery: return run_grouped(k_query_group, q, st);
    case kRouteQueryMid: return run_grouped(k_query_mid_group, q, st);
    case kRouteB2List: return run_grouped(k_b2list_group, q, st);
    case kRouteBrute: return run_grouped(k_brute_group, q, st, 0);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_route_sparse_sites(const RouteArgs& a, cudaStream_t st)
{
    return a.rank == 3 ? launch_chained(k_b2sparse<3>, dim3(resident(k_b2sparse<3>)), dim3(256), 0, st, a)
                       : launch_chained(k_b2sparse<2>, dim3(resident(k_b2sparse<2>)), dim3(256), 0, st, a);
}

}  // namespace qai
