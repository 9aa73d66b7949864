// qai_local.cu -- the local first EDT: steps A, B and C of Algorithm 4 for
// fields whose quantization boundary is dense.
//
// Step B needs, at every point, the nearest point of B1 (Eq. 2) with the
// smallest linear index among equally near ones (the tie rule of the
// separable passes of Algorithm 1), and step C its sign S = S_B[I1]
// (Algorithm 3). Where B1 is dense -- a rough field or a small error bound,
// where almost every point differs from a neighbour -- the nearest site is a
// few cells away, and a bounded search finds it exactly:
//
//   k_detect  step A (Algorithm 2) at every point: the equal-q mask with the
//             sign code of S_B packed in (a point is on B1 iff it is interior
//             and some neighbour differs; points off the interior get the
//             all-equal mask), the output wherever Dist2 does not matter
//             (D' + S_B eta eps on B1, D' elsewhere), and the list of B1
//             points with S != 0. Dist1 = 0 on B1 is not stored: readers take
//             B1 from the mask byte.
//   k_near    every point off B1 scans the lattice offsets of squared length
//             <= 8 in order of (squared length, dz, dy, dx) -- for points
//             inside the field that is the order of (distance, linear index)
//             -- and takes the first B1 point it meets: Dist1 and I1 exactly,
//             since any point outside that ball is at squared distance >= 9.
//             It writes S everywhere, Dist1 where S != 0, and lists the
//             queries of the second EDT (S != 0 off B1). k_near_sparse does
//             the same for rows of 16-byte multiples, with the search run
//             only on the 4-point words that hold a point off B1, gathered
//             across the warp.
//
// A point with no B1 point within that ball sets kCtrLocalFail; the separable
// first EDT (row pass 1, column passes 1) then runs and rewrites all of it.
#include "qai_detect.cuh"
#include "qai_device.cuh"
#include "qai_launch.h"

namespace qai {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Offsets of squared length 1..8, sorted by (r2, dz, dy, dx): (r2 << 24) |
// (dz & 0xFF) << 16 | (dy & 0xFF) << 8 | (dx & 0xFF). near3 spans three axes,
// near2 two (dz = 0).
constexpr int kNearR2 = 8;
constexpr int kNearN3 = 92, kNearN2 = 24;
struct NearTable {
    int off3[kNearN3];
    int off2[kNearN2];
};
constexpr int pack_near(int r2, int dz, int dy, int dx)
{
    return (int)(((unsigned)r2 << 24) | ((unsigned)(dz & 0xFF) << 16) | ((unsigned)(dy & 0xFF) << 8) |
                 (unsigned)(dx & 0xFF));
}
constexpr NearTable make_near()
{
    NearTable t{};
    int n3 = 0, n2 = 0;
    for (int r2 = 1; r2 <= kNearR2; ++r2)
        for (int dz = -2; dz <= 2; ++dz)
            for (int dy = -2; dy <= 2; ++dy)
                for (int dx = -2; dx <= 2; ++dx)
                    if (dz * dz + dy * dy + dx * dx == r2) {
                        t.off3[n3++] = pack_near(r2, dz, dy, dx);
                        if (dz == 0) t.off2[n2++] = pack_near(r2, 0, dy, dx);
                    }
    return t;
}
constexpr int count_near(bool three)
{
    int n = 0;
    for (int dz = three ? -2 : 0; dz <= (three ? 2 : 0); ++dz)
        for (int dy = -2; dy <= 2; ++dy)
            for (int dx = -2; dx <= 2; ++dx)
                if (dz * dz + dy * dy + dx * dx >= 1 && dz * dz + dy * dy + dx * dx <= kNearR2) ++n;
    return n;
}
static_assert(count_near(true) == kNearN3 && count_near(false) == kNearN2, "nearest-site table size");
__constant__ NearTable c_near = make_near();

// Minimum resident CTAs per SM the kernels are compiled for (register cap).
#ifndef QAI_DETECT_MINB
#define QAI_DETECT_MINB 5
#endif
#ifndef QAI_NEAR_MINB
#define QAI_NEAR_MINB 5
#endif
// Grid of the step-A kernel in resident waves.
#ifndef QAI_DETECT_WAVES
#define QAI_DETECT_WAVES 2
#endif

// Per-CTA collection of list entries before one global atomic per CTA.
constexpr int kSignedCta = 1024;
constexpr int kQueryCta = 2048;

// Step A on one warp-segment of 128 points (4 per lane) of row `row`.
// The q values one lane needs for its four points of a segment: the row and
// its four neighbour rows (zeros off the interior rows), and the value next
// to the segment for the first lane (x0 - 1) and the last (x0 + 4).
struct SegQ {
    int c[4], yl[4], yr[4], zl[4], zr[4];
    int edge;
};

template <int RANK, bool VEC>
__device__ __forceinline__ void load_segment(const LocalArgs& a, int row, int z, int y, int x0, SegQ& L)
{
    const int lane = threadIdx.x & 31;
    const int nx = a.nx;
    const int rbase = row * nx;
    const int plane = a.ny * nx;
    const bool row_inner = y >= 1 && y <= a.ny - 2 && (RANK == 2 || (z >= 1 && z <= a.nz - 2));
    load4_i32(a.q + rbase, x0, nx, VEC, L.c);
#pragma unroll
    for (int j = 0; j < 4; ++j) L.yl[j] = L.yr[j] = L.zl[j] = L.zr[j] = 0;
    if (row_inner) {
        load4_i32(a.q + rbase - nx, x0, nx, VEC, L.yl);
        load4_i32(a.q + rbase + nx, x0, nx, VEC, L.yr);
        if (RANK == 3) {
            load4_i32(a.q + rbase - plane, x0, nx, VEC, L.zl);
            load4_i32(a.q + rbase + plane, x0, nx, VEC, L.zr);
        }
    }
    L.edge = 0;
    if (lane == 0 && x0 > 0) L.edge = __ldg(a.q + rbase + x0 - 1);
    if (lane == 31 && x0 + 4 < nx) L.edge = __ldg(a.q + rbase + x0 + 4);
}

template <int RANK, bool VEC>
__device__ __forceinline__ void detect_segment(const LocalArgs& a, int row, int z, int y, int x0, const SegQ& L,
                                               int32_t* sbuf, int* sn)
{
    const int lane = threadIdx.x & 31;
    const int nx = a.nx;
    const int rbase = row * nx;
    const bool row_inner = y >= 1 && y <= a.ny - 2 && (RANK == 2 || (z >= 1 && z <= a.nz - 2));
    const int *c = L.c, *yl = L.yl, *yr = L.yr, *zl = L.zl, *zr = L.zr;
    int xm = __shfl_up_sync(kFull, c[3], 1);
    int xp = __shfl_down_sync(kFull, c[0], 1);
    if (lane == 0) xm = L.edge;
    if (lane == 31) xp = L.edge;
    unsigned em = 0x3F3F3F3Fu;  // all equal: off the interior nothing is on B1
    unsigned codes = 0;         // 2-bit sign code of S_B per point (B1 points only)
    if (row_inner) {            // warp-uniform
        // 32-bit sums are exact while every |q| < 2^27; OR of the raw values
        // is below 2^27 exactly when all are in [0, 2^27), the common case
        unsigned acc = (unsigned)xm | (unsigned)xp;
#pragma unroll
        for (int j = 0; j < 4; ++j) acc |= (unsigned)c[j] | (unsigned)yl[j] | (unsigned)yr[j] | (unsigned)zl[j] | (unsigned)zr[j];
        bool narrow = acc < (1u << 27);
        if (!__all_sync(kFull, narrow)) {
            acc = (unsigned)(xm ^ (xm >> 31)) | (unsigned)(xp ^ (xp >> 31));
#pragma unroll
            for (int j = 0; j < 4; ++j)
                acc |= (unsigned)(c[j] ^ (c[j] >> 31)) | (unsigned)(yl[j] ^ (yl[j] >> 31)) |
                       (unsigned)(yr[j] ^ (yr[j] >> 31)) | (unsigned)(zl[j] ^ (zl[j] >> 31)) |
                       (unsigned)(zr[j] ^ (zr[j] >> 31));
            narrow = acc < (1u << 27);
        }
        const bool wide = __any_sync(kFull, !narrow);
        // interior along x: only the first and the last lanes of a row have
        // points off it
        const unsigned inner_bits = (x0 >= 1 && x0 + 4 <= nx - 1)
                                        ? 0xFu
                                        : ((x0 >= 1 && x0 <= nx - 2) ? 1u : 0u) | ((x0 + 1 >= 1 && x0 + 1 <= nx - 2) ? 2u : 0u) |
                                              ((x0 + 2 <= nx - 2) ? 4u : 0u) | ((x0 + 3 <= nx - 2) ? 8u : 0u);
        em = 0;
        if (!wide && a.m.sign_rule == 0) {
            // the common case in two steps: masks and the fast-varying test
            // at every point, the sign only where a boundary keeps it
            const int thm1 = a.m.grad_threshold - 1;
            const unsigned lim = 2u * (unsigned)thm1;
            unsigned keep = 0;  // bit j: point j is on B1 and not fast-varying
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q0 = c[j];
                const int l = j == 0 ? xm : c[j - 1];
                const int r = j == 3 ? xp : c[j + 1];
                // differing-neighbour bits: min(n ^ q0, 1) is 1 exactly where
                // n != q0; the mask byte keeps the complement (equal bits)
                unsigned ne = umin((unsigned)(l ^ q0), 1u) * 0x10u + umin((unsigned)(r ^ q0), 1u) * 0x20u;
                bool fast = (unsigned)(r - l + thm1) > lim;
                ne += umin((unsigned)(yl[j] ^ q0), 1u) * 0x4u + umin((unsigned)(yr[j] ^ q0), 1u) * 0x8u;
                fast |= (unsigned)(yr[j] - yl[j] + thm1) > lim;
                if (RANK == 3) {
                    ne += umin((unsigned)(zl[j] ^ q0), 1u) + umin((unsigned)(zr[j] ^ q0), 1u) * 0x2u;
                    fast |= (unsigned)(zr[j] - zl[j] + thm1) > lim;
                }
                const bool inner = (inner_bits >> j) & 1u;
                keep |= (inner && ne != 0u && !fast) ? 1u << j : 0u;
                em |= (0x3Fu ^ (inner ? ne : 0u)) << (8 * j);
            }
            if (__any_sync(kFull, keep != 0)) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!((keep >> j) & 1u)) continue;
                    const int l = j == 0 ? xm : c[j - 1];
                    const int r = j == 3 ? xp : c[j + 1];
                    int sum = l + r + yl[j] + yr[j] - 2 * RANK * c[j];
                    if (RANK == 3) sum += zl[j] + zr[j];
                    const unsigned cd = sum > 0 ? 1u : (sum < 0 ? 2u : 0u);
                    em |= cd << (8 * j + 6);
                    codes |= cd << (2 * j);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool inner = (inner_bits >> j) & 1u;
                const int l = j == 0 ? xm : c[j - 1];
                const int r = j == 3 ? xp : c[j + 1];
                unsigned mk;
                bool site;
                int code;
                if (!wide) detect_point<RANK, false>(c[j], zl[j], zr[j], yl[j], yr[j], l, r, inner, a.m, mk, site, code);
                else detect_point<RANK, true>(c[j], zl[j], zr[j], yl[j], yr[j], l, r, inner, a.m, mk, site, code);
                const unsigned cd = (unsigned)code;  // 0 off the interior
                em |= ((inner ? mk : 0x3Fu) | cd << 6) << (8 * j);
                codes |= cd << (2 * j);
            }
        }
    }
    // outputs where Dist2 does not matter: the expressions of compensate()
    // (with C = +0 the fma is the product)
    float o[4];
    if (__any_sync(kFull, codes != 0)) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned cd = (codes >> (2 * j)) & 3u;
            const float cc = (cd == 1u ? 1.0f : (cd == 2u ? -1.0f : 0.0f)) * a.m.eta_eb;
            o[j] = a.m.output_c ? cc : fmaf((float)c[j], a.m.two_eb, cc);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = a.m.output_c ? 0.0f : (float)c[j] * a.m.two_eb;
    }
    if (VEC) {
        if (x0 < nx) {
            *reinterpret_cast<uint32_t*>(a.eqm + rbase + x0) = em;
            *reinterpret_cast<float4*>(a.out + rbase + x0) = make_float4(o[0], o[1], o[2], o[3]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (x0 + j < nx) {
                a.eqm[rbase + x0 + j] = (uint8_t)(em >> (8 * j));
                a.out[rbase + x0 + j] = o[j];
            }
    }
    // B1 points with S != 0: the signed set lists them (Dist1 = 0 there is
    // not stored; the mask byte tells B1), until the CTA's buffer is full
    if (codes && *static_cast<volatile int*>(sn) <= kSignedCta) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (((codes >> (2 * j)) & 3u) == 0u) continue;
            const int k = atomicAdd(sn, 1);
            if (k < kSignedCta) sbuf[k] = rbase + x0 + j;
        }
    }
}

template <int RANK, bool VEC>
__global__ void __launch_bounds__(256, QAI_DETECT_MINB) k_detect(LocalArgs a)
{
    wait_prior_grid();
    __shared__ int32_t sbuf[kSignedCta];
    __shared__ int sn, sbase;
    if (threadIdx.x == 0) sn = 0;
    __syncthreads();
    const int rows = a.nz * a.ny;
    const int wstride = gridDim.x * (blockDim.x >> 5);
    const int lx = 4 * (int)(threadIdx.x & 31);
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += wstride) {
        const int z = RANK == 3 ? row / a.ny : 0;
        const int y = row - z * a.ny;
        for (int x0 = lx; x0 - lx < a.nx; x0 += 128) {
            SegQ b;
            load_segment<RANK, VEC>(a, row, z, y, x0, b);
            detect_segment<RANK, VEC>(a, row, z, y, x0, b, sbuf, &sn);
        }
    }

    __syncthreads();
    const int n = sn;
    if (threadIdx.x == 0) {
        sbase = -1;
        if (n > kSignedCta) *static_cast<volatile int*>(a.ctr + kCtrSignedOver) = 1;
        else if (n > 0) sbase = atomicAdd(a.ctr + kCtrSigned, n);
    }
    __syncthreads();
    if (sbase >= 0)
        for (int i = threadIdx.x; i < n && sbase + i < a.scap; i += blockDim.x) a.slist[sbase + i] = sbuf[i];
}

// The nearest B1 point of p (off B1): its squared distance and the sign code
// it carries, or r2 = -1 when none lies within squared distance 8.
// The nearest B1 point of p (off B1) among table entries k0.. (the first 6,
// or 4 in 2-D, are the squared distance 1): its squared distance and the sign
// code it carries, or r2 = -1 when none lies within squared distance 8. The table is scanned in chunks of eight entries whose
// loads are issued together; the first B1 point in table order is the answer.
template <int RANK>
__device__ __forceinline__ void nearest_site(const LocalArgs& a, int p, int z, int y, int x, int k0, int& r2,
                                             unsigned& code)
{
    const int plane = a.ny * a.nx;
    const int* tab = RANK == 3 ? c_near.off3 : c_near.off2;
    constexpr int ntab = RANK == 3 ? kNearN3 : kNearN2;
    r2 = -1;
    code = 0;
    for (; k0 < ntab; k0 += 8) {
        unsigned e[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            e[u] = 0x3Fu;
            const int k = k0 + u;
            if (k >= ntab) continue;
            const int o = tab[k];
            const int dx = (int)(int8_t)(o & 0xFF), dy = (int)(int8_t)((o >> 8) & 0xFF);
            const int dz = (int)(int8_t)((o >> 16) & 0xFF);
            const bool in = (unsigned)(x + dx) < (unsigned)a.nx && (unsigned)(y + dy) < (unsigned)a.ny &&
                            (RANK == 2 || (unsigned)(z + dz) < (unsigned)a.nz);
            if (in) e[u] = __ldg(a.eqm + p + dz * plane + dy * a.nx + dx);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (k0 + u < ntab && (e[u] & 0x3Fu) != 0x3Fu) {
                r2 = (int)((unsigned)tab[k0 + u] >> 24);
                code = e[u] >> 6;
                return;
            }
        }
    }
}

// Four bytes of a row at x0.. (0x3F, "not on B1", past the row end).
__device__ __forceinline__ uint32_t load4_em(const uint8_t* row, int x0, int nx, bool vec)
{
    if (vec) return x0 < nx ? __ldg(reinterpret_cast<const uint32_t*>(row + x0)) : 0x3F3F3F3Fu;
    uint32_t w = 0x3F3F3F3Fu;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (x0 + j < nx) w = (w & ~(0xFFu << (8 * j))) | (uint32_t)__ldg(row + x0 + j) << (8 * j);
    return w;
}

// Byte k = 0xFF where byte k of the mask word marks a B1 point (some of its
// six equal-q bits clear): t = the clear bits, at most 0x3F per byte, so
// t + 0x7F sets bit 7 of a byte exactly when t is not zero, with no carry;
// the byte permute with selector nibbles 8..B copies each byte's bit 7 over
// the byte.
__device__ __forceinline__ uint32_t site_bytes(uint32_t w)
{
    const uint32_t t = (~w & 0x3F3F3F3Fu) + 0x7F7F7F7Fu;
    uint32_t r;
    asm("prmt.b32 %0, %1, 0, 0xBA98;" : "=r"(r) : "r"(t));  // sign-replicating byte permute
    return r;
}

// S bytes of the four points xk .. xk + 3 of row `row`, with Dist1 and the
// query-list entries of those that are queries (S != 0 off B1). cw holds
// their mask bytes, pw and nw the words either side (for the x - 1 and x + 1
// neighbours), ylw .. zrw the words of the four neighbour rows (0x3F: no
// point). The six neighbours at squared distance 1 are tested for the four
// points at once, byte-wise, in the tie order z-, y-, x-, x+, y+, z+
// (increasing linear index); a point with none of them on B1 scans the rest
// of the table alone.
template <int RANK>
__device__ __forceinline__ uint32_t near_word(const LocalArgs& a, int row, int z, int y, int xk, uint32_t cw,
                                              uint32_t pw, uint32_t nw, uint32_t ylw, uint32_t yrw, uint32_t zlw,
                                              uint32_t zrw, Query* qbuf, int* qn, bool& fail)
{
    const uint32_t own = site_bytes(cw), pm = site_bytes(pw), nm = site_bytes(nw);
    const uint32_t xlw = __byte_perm(pw, cw, 0x6543), xlm = __byte_perm(pm, own, 0x6543);  // x - 1
    const uint32_t xrw = __byte_perm(cw, nw, 0x4321), xrm = __byte_perm(own, nm, 0x4321);  // x + 1
    // the first B1 neighbour in tie order: select from the last to the first
    uint32_t found = 0, pick = 0x3F3F3F3Fu;
    auto take = [&](uint32_t w, uint32_t m) {
        pick = (w & m) | (pick & ~m);
        found |= m;
    };
    take(zrw, site_bytes(zrw));
    take(yrw, site_bytes(yrw));
    take(xrw, xrm);
    take(xlw, xlm);
    take(ylw, site_bytes(ylw));
    take(zlw, site_bytes(zlw));
    // codes: own on B1, else the neighbour's; Dist1 = 1 where resolved off
    // B1 (bytes past the row end, and x - 1 of x = 0, read 0x3F)
    const int nvalid = min(4, a.nx - xk);
    const uint32_t valid = nvalid >= 4 ? 0xFFFFFFFFu : (nvalid <= 0 ? 0u : (1u << (8 * nvalid)) - 1u);
    uint32_t cw2 = ((own & cw) | (~own & pick)) >> 6 & 0x03030303u;
    const uint32_t need = ~own & ~found & valid;  // no site within r2 = 1: scan the table
    uint32_t d1w = ~own & 0x01010101u;
    if (need) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!((need >> (8 * j)) & 0xFFu)) continue;
            int r2;
            unsigned code;
            nearest_site<RANK>(a, row * a.nx + xk + j, z, y, xk + j, RANK == 3 ? 6 : 4, r2, code);
            if (r2 < 0) {
                fail = true;
                r2 = 0;
                code = 0;
            }
            cw2 = (cw2 & ~(0xFFu << (8 * j))) | code << (8 * j);
            d1w = (d1w & ~(0xFFu << (8 * j))) | (uint32_t)r2 << (8 * j);
        }
    }
    // S bytes: code 1 -> +1, code 2 -> -1
    const uint32_t pos = cw2 & 0x01010101u, neg = (cw2 >> 1) & 0x01010101u;
    // queries: S != 0 off B1
    const uint32_t qmask = (pos | neg) & ~own & valid;
    if (qmask) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!((qmask >> (8 * j)) & 1u)) continue;
            const int p = row * a.nx + xk + j;
            const int r2 = (int)((d1w >> (8 * j)) & 0xFFu);
            const unsigned code = (cw2 >> (8 * j)) & 3u;
            a.dist1[p] = r2;
            const Query qe{p, (r2 << 2) | (int)code};
            const int kq = atomicAdd(qn, 1);
            if (kq < kQueryCta) {
                qbuf[kq] = qe;
            } else {
                const int g = atomicAdd(a.ctr + kCtrQueries, 1);
                if (g < a.qcap) a.qlist[g] = qe;
            }
        }
    }
    return pos | (neg * 0xFFu);
}

// The CTA's queries to the global list (one atomic), and the flag of a point
// with no B1 point within reach.
__device__ __forceinline__ void near_flush(const LocalArgs& a, const Query* qbuf, const int* qn, int* qbase, bool fail)
{
    if (__any_sync(kFull, fail) && (threadIdx.x & 31) == 0) *static_cast<volatile int*>(a.ctr + kCtrLocalFail) = 1;
    __syncthreads();
    const int n = min(*qn, kQueryCta);
    if (threadIdx.x == 0) *qbase = n > 0 ? atomicAdd(a.ctr + kCtrQueries, n) : 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n && *qbase + i < a.qcap; i += blockDim.x) a.qlist[*qbase + i] = qbuf[i];
}

// S at every point, Dist1 where S != 0 off B1, and the queries, for rows of
// any length: one warp per row, four points per lane and step.
template <int RANK>
__global__ void __launch_bounds__(256, QAI_NEAR_MINB) k_near(LocalArgs a)
{
    wait_prior_grid();
    __shared__ Query qbuf[kQueryCta];
    __shared__ int qn, qbase;
    if (threadIdx.x == 0) qn = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int rows = a.nz * a.ny;
    const int plane = a.ny * a.nx;
    const int wstride = gridDim.x * (blockDim.x >> 5);
    bool fail = false;
    const uint32_t none = 0x3F3F3F3Fu;
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += wstride) {
        const int z = RANK == 3 ? row / a.ny : 0;
        const int y = row - z * a.ny;
        const uint8_t* er = a.eqm + (int64_t)row * a.nx;
        int8_t* sr = a.s + (int64_t)row * a.nx;
        uint32_t carry = none;  // the word of the previous step (its byte 3 is x - 1 of byte 0)
        for (int xs = 0; xs < a.nx; xs += 128) {
            const int x0 = xs + 4 * lane;
            const uint32_t cw = load4_em(er, x0, a.nx, false);
            const uint32_t ylw = y > 0 ? load4_em(er - a.nx, x0, a.nx, false) : none;
            const uint32_t yrw = y < a.ny - 1 ? load4_em(er + a.nx, x0, a.nx, false) : none;
            const uint32_t zlw = RANK == 3 && z > 0 ? load4_em(er - plane, x0, a.nx, false) : none;
            const uint32_t zrw = RANK == 3 && z < a.nz - 1 ? load4_em(er + plane, x0, a.nx, false) : none;
            uint32_t prev = __shfl_up_sync(kFull, cw, 1);
            uint32_t next = __shfl_down_sync(kFull, cw, 1);
            const uint32_t last = __shfl_sync(kFull, cw, 31);
            if (lane == 0) prev = carry;
            if (lane == 31) next = x0 + 4 < a.nx ? (uint32_t)__ldg(er + x0 + 4) : 0x3Fu;
            carry = last;
            const uint32_t sw = near_word<RANK>(a, row, z, y, x0, cw, prev, next, ylw, yrw, zlw, zrw, qbuf, &qn, fail);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x0 + j < a.nx) sr[x0 + j] = (int8_t)(sw >> (8 * j));
        }
    }
    near_flush(a, qbuf, &qn, &qbase, fail);
}

// The same for rows of 16-byte multiples, sparse in the points off B1 (most
// points of a field with a dense B1 are on it and keep their own sign). A
// lane reads 16 mask bytes of the row per step (one 128-bit load) and writes
// the S of its B1 points; the words holding a point off B1 are gathered
// across the warp (a ballot per word position) and dealt one per lane to
// near_word, which reads the neighbour words it needs. The S words meet in
// shared memory before the lane's 128-bit store.
template <int RANK>
__global__ void __launch_bounds__(256, QAI_NEAR_MINB) k_near_sparse(LocalArgs a)
{
    wait_prior_grid();
    __shared__ Query qbuf[kQueryCta];
    __shared__ uint32_t swb[8][4 * 32];
    __shared__ int qn, qbase;
    if (threadIdx.x == 0) qn = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint32_t* sw = swb[threadIdx.x >> 5];  // word k of lane l at [32 k + l]
    const int rows = a.nz * a.ny;
    const int plane = a.ny * a.nx;
    const int wstride = gridDim.x * (blockDim.x >> 5);
    bool fail = false;
    const uint32_t none = 0x3F3F3F3Fu;
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += wstride) {
        const int z = RANK == 3 ? row / a.ny : 0;
        const int y = row - z * a.ny;
        const uint8_t* er = a.eqm + (int64_t)row * a.nx;
        int8_t* sr = a.s + (int64_t)row * a.nx;
        for (int xs = 0; xs < a.nx; xs += 512) {
            const int x0 = xs + 16 * lane;
            const bool in = x0 < a.nx;  // rows are 16-byte multiples: four words or none
            const uint4 c = in ? __ldg(reinterpret_cast<const uint4*>(er + x0)) : make_uint4(none, none, none, none);
            unsigned off[4];  // word position k: the lanes whose word k holds a point off B1
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t cw = k == 0 ? c.x : (k == 1 ? c.y : (k == 2 ? c.z : c.w));
                const uint32_t own = site_bytes(cw);
                const uint32_t cw2 = (own & cw) >> 6 & 0x03030303u;  // B1 points: their own code
                const uint32_t pos = cw2 & 0x01010101u, neg = (cw2 >> 1) & 0x01010101u;
                sw[32 * k + lane] = pos | (neg * 0xFFu);
                off[k] = __ballot_sync(kFull, in && own != 0xFFFFFFFFu);
            }
            const int n0 = __popc(off[0]), n1 = __popc(off[1]), n2 = __popc(off[2]), n3 = __popc(off[3]);
            const int total = n0 + n1 + n2 + n3;
            __syncwarp();
            for (int e = lane; e - lane < total; e += 32) {
                if (e >= total) continue;
                int k, r;
                if (e < n0) {
                    k = 0; r = e;
                } else if (e < n0 + n1) {
                    k = 1; r = e - n0;
                } else if (e < n0 + n1 + n2) {
                    k = 2; r = e - n0 - n1;
                } else {
                    k = 3; r = e - n0 - n1 - n2;
                }
                const unsigned bk = k == 0 ? off[0] : (k == 1 ? off[1] : (k == 2 ? off[2] : off[3]));
                const int src = (int)__fns(bk, 0, r + 1);  // the lane that holds the word
                const int xk = xs + 16 * src + 4 * k;
                auto w32 = [&](const uint8_t* rp) { return __ldg(reinterpret_cast<const uint32_t*>(rp + xk)); };
                const uint32_t cw = w32(er);
                const uint32_t pw = xk >= 4 ? w32(er - 4) : none;
                const uint32_t nw = xk + 4 < a.nx ? w32(er + 4) : none;
                const uint32_t ylw = y > 0 ? w32(er - a.nx) : none;
                const uint32_t yrw = y < a.ny - 1 ? w32(er + a.nx) : none;
                const uint32_t zlw = RANK == 3 && z > 0 ? w32(er - plane) : none;
                const uint32_t zrw = RANK == 3 && z < a.nz - 1 ? w32(er + plane) : none;
                sw[32 * k + src] = near_word<RANK>(a, row, z, y, xk, cw, pw, nw, ylw, yrw, zlw, zrw, qbuf, &qn, fail);
            }
            __syncwarp();
            if (in)
                *reinterpret_cast<uint4*>(sr + x0) = make_uint4(sw[lane], sw[32 + lane], sw[64 + lane], sw[96 + lane]);
            __syncwarp();
        }
    }
    near_flush(a, qbuf, &qn, &qbase, fail);
}

}  // namespace

namespace {
// A grid-stride kernel's grid: every CTA resident at once (one wave).
template <class K>
int one_wave(K kern, int waves = 1)
{
    int dev = 0, sms = 152, per = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0) != cudaSuccess || per < 1) per = 1;
    return sms * per * waves;
}
}  // namespace

cudaError_t launch_local_detect(const LocalArgs& a, cudaStream_t st)
{
    auto run = [&](auto kern) {
        return launch_chained(kern, dim3(one_wave(kern, QAI_DETECT_WAVES)), dim3(256), 0, st, a);
    };
    if (a.rank == 3) return a.vec ? run(k_detect<3, true>) : run(k_detect<3, false>);
    return a.vec ? run(k_detect<2, true>) : run(k_detect<2, false>);
}

cudaError_t launch_local_near(const LocalArgs& a, cudaStream_t st)
{
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const bool wide = (a.nx % 16 == 0) && al(a.eqm) && al(a.s);  // 16-byte rows
    auto run = [&](auto kern) {
        return launch_chained(kern, dim3(one_wave(kern)), dim3(256), 0, st, a);
    };
    if (a.rank == 3) return wide ? run(k_near_sparse<3>) : run(k_near<3>);
    return wide ? run(k_near_sparse<2>) : run(k_near<2>);
}

}  // namespace qai
