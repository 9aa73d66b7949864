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
//   k_detect  step A (Algorithm 2) at every point: whether the point is on B1
//             (interior, some axis neighbour differs) and the sign code of
//             S_B, as a 2-bit code per point in the packed `codes` map; the
//             output wherever Dist2 does not matter (D' + S_B eta eps on B1,
//             D' elsewhere); the count of B1 points with S != 0. It reads q
//             once and writes 4.25 bytes per point.
//   k_near    S at every point into the packed `spk` map. A point on B1
//             keeps S_B. A point off B1 takes the first B1 point among the
//             lattice offsets of squared length <= 8 in order of (squared
//             length, dz, dy, dx) -- for points inside the field that is the
//             order of (distance, linear index) -- which gives Dist1 and I1
//             exactly, since any point outside that ball is at squared
//             distance >= 9. The search runs on 16 points at once, on the
//             2-bit fields of one word: for each offset the neighbour word is
//             shifted into place and the still-unresolved fields with a site
//             there take its code. Queries of the second EDT (S != 0 off B1)
//             go to the query list with Dist1.
//
// A point with no B1 point within that ball sets kCtrLocalFail; the separable
// first EDT (row pass 1, column passes 1) then runs and rewrites all of it,
// and k_pack_s packs its S map for the route. k_expand writes the byte maps
// (equal-q mask, S) that the separable second EDT and the adjoint read.
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

// First table entry of squared length r2 (1..9: one past the table for 9),
// 3-D or 2-D table.
constexpr int group_begin(bool three, int r2)
{
    int k = 0;
    for (int dz = three ? -2 : 0; dz <= (three ? 2 : 0); ++dz)
        for (int dy = -2; dy <= 2; ++dy)
            for (int dx = -2; dx <= 2; ++dx) {
                const int d = dz * dz + dy * dy + dx * dx;
                if (d >= 1 && d <= kNearR2 && d < r2) ++k;
            }
    return k;
}
static_assert(group_begin(true, 2) == 6 && group_begin(false, 2) == 4 && group_begin(true, 9) == kNearN3 &&
                  group_begin(false, 9) == kNearN2,
              "nearest-site table groups");

// Minimum resident CTAs per SM the kernels are compiled for (register cap).
#ifndef QAI_DETECT_MINB
#define QAI_DETECT_MINB 5
#endif
#ifndef QAI_NEAR_MINB
#define QAI_NEAR_MINB 4
#endif
// Grid of the step-A kernel in resident waves.
#ifndef QAI_DETECT_WAVES
#define QAI_DETECT_WAVES 2
#endif

// Per-CTA collection of query-list entries before one global atomic per CTA.
constexpr int kQueryCta = 2048;

// The low bit of every nonzero 2-bit field of v.
__device__ __forceinline__ uint32_t field_lsb(uint32_t v) { return (v | (v >> 1)) & 0x55555555u; }

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
    const int64_t rbase = (int64_t)row * nx;
    const int64_t plane = (int64_t)a.ny * nx;
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

// Step A for the lane's four points: b1 (bit j: point j on B1), sg (2-bit
// sign code of S_B per point, 0 off B1) and, when MASK, the equal-q mask
// byte per point (the byte map of the separable passes: bits z-, z+, y-, y+,
// x-, x+, 0x3F off the interior).
template <int RANK, bool MASK>
__device__ __forceinline__ void step_a(const LocalArgs& a, int z, int y, int x0, const SegQ& L, unsigned& b1,
                                       unsigned& sg, uint32_t& em)
{
    const int lane = threadIdx.x & 31;
    const int nx = a.nx;
    const bool row_inner = y >= 1 && y <= a.ny - 2 && (RANK == 2 || (z >= 1 && z <= a.nz - 2));
    const int *c = L.c, *yl = L.yl, *yr = L.yr, *zl = L.zl, *zr = L.zr;
    int xm = __shfl_up_sync(kFull, c[3], 1);
    int xp = __shfl_down_sync(kFull, c[0], 1);
    if (lane == 0) xm = L.edge;
    if (lane == 31) xp = L.edge;
    b1 = 0;
    sg = 0;
    em = 0x3F3F3F3Fu;
    if (!row_inner) return;  // warp-uniform: off the interior nothing is on B1
    // 32-bit sums are exact while every |q| < 2^27; the OR of the raw values
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
    if (!MASK && !wide && a.m.sign_rule == 0) {
        // the common case in two steps: B1 and the fast-varying test at
        // every point, the sign only where a boundary keeps it
        const int thm1 = a.m.grad_threshold - 1;
        const unsigned lim = 2u * (unsigned)thm1;
        unsigned keep = 0;  // bit j: point j is on B1 and not fast-varying
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q0 = c[j];
            const int l = j == 0 ? xm : c[j - 1];
            const int r = j == 3 ? xp : c[j + 1];
            unsigned d = ((unsigned)l ^ (unsigned)q0) | ((unsigned)r ^ (unsigned)q0) |
                         ((unsigned)yl[j] ^ (unsigned)q0) | ((unsigned)yr[j] ^ (unsigned)q0);
            bool fast = (unsigned)(r - l + thm1) > lim || (unsigned)(yr[j] - yl[j] + thm1) > lim;
            if (RANK == 3) {
                d |= ((unsigned)zl[j] ^ (unsigned)q0) | ((unsigned)zr[j] ^ (unsigned)q0);
                fast = fast || (unsigned)(zr[j] - zl[j] + thm1) > lim;
            }
            const bool site = ((inner_bits >> j) & 1u) && d != 0u;
            b1 |= site ? 1u << j : 0u;
            keep |= (site && !fast) ? 1u << j : 0u;
        }
        if (__any_sync(kFull, keep != 0)) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!((keep >> j) & 1u)) continue;
                const int l = j == 0 ? xm : c[j - 1];
                const int r = j == 3 ? xp : c[j + 1];
                int sum = l + r + yl[j] + yr[j] - 2 * RANK * c[j];
                if (RANK == 3) sum += zl[j] + zr[j];
                sg |= (sum > 0 ? 1u : (sum < 0 ? 2u : 0u)) << (2 * j);
            }
        }
        return;
    }
    em = 0;
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
        b1 |= site ? 1u << j : 0u;
        sg |= (unsigned)code << (2 * j);  // 0 off the interior
        em |= ((inner ? mk : 0x3Fu) | (unsigned)code << 6) << (8 * j);
    }
}

// Bits 0, 1, 2, 3 of b to bits 0, 2, 4, 6.
__device__ __forceinline__ unsigned spread4(unsigned b)
{
    return (b & 1u) | ((b & 2u) << 1) | ((b & 4u) << 2) | ((b & 8u) << 3);
}

template <int RANK, bool VEC>
__device__ __forceinline__ void detect_segment(const LocalArgs& a, int row, int z, int y, int x0, const SegQ& L,
                                               unsigned& nsigned)
{
    const int nx = a.nx;
    const int64_t rbase = (int64_t)row * nx;
    unsigned b1, sg;
    uint32_t em;
    step_a<RANK, false>(a, z, y, x0, L, b1, sg, em);
    // outputs where Dist2 does not matter: the expressions of compensate()
    // (with C = +0 the fma is the product)
    float o[4];
    if (__any_sync(kFull, sg != 0)) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned cd = (sg >> (2 * j)) & 3u;
            const float cc = (cd == 1u ? 1.0f : (cd == 2u ? -1.0f : 0.0f)) * a.m.eta_eb;
            o[j] = a.m.output_c ? cc : fmaf((float)L.c[j], a.m.two_eb, cc);
        }
        nsigned += __popc(field_lsb(sg));
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = a.m.output_c ? 0.0f : (float)L.c[j] * a.m.two_eb;
    }
    if (VEC) {
        if (x0 < nx) *reinterpret_cast<float4*>(a.out + rbase + x0) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (x0 + j < nx) a.out[rbase + x0 + j] = o[j];
    }
    // the code byte of the four points (0 past nx, up to the row's last word)
    if (x0 < 16 * a.wpr)
        reinterpret_cast<uint8_t*>(a.codes)[(int64_t)row * 4 * a.wpr + (x0 >> 2)] = (uint8_t)(spread4(b1) + sg);
}

template <int RANK, bool VEC>
__global__ void __launch_bounds__(256, QAI_DETECT_MINB) k_detect(LocalArgs a)
{
    wait_prior_grid();
    const int rows = a.nz * a.ny;
    const int wstride = gridDim.x * (blockDim.x >> 5);
    const int lx = 4 * (int)(threadIdx.x & 31);
    unsigned nsigned = 0;
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += wstride) {
        const int z = RANK == 3 ? row / a.ny : 0;
        const int y = row - z * a.ny;
        for (int x0 = lx; x0 - lx < a.nx; x0 += 128) {
            SegQ b;
            load_segment<RANK, VEC>(a, row, z, y, x0, b);
            detect_segment<RANK, VEC>(a, row, z, y, x0, b, nsigned);
        }
    }
    // B1 points with S != 0: one atomic per warp that has any
    nsigned = __reduce_add_sync(kFull, nsigned);
    if ((threadIdx.x & 31) == 0 && nsigned) atomicAdd(a.ctr + kCtrSigned, (int)nsigned);
}

// Word k of packed row `prow` (0 past the row, or where ok is false).
__device__ __forceinline__ uint32_t pword(const uint32_t* m, int64_t prow, int k, int wpr, bool ok)
{
    return ok && k >= 0 && k < wpr ? __ldg(m + prow * wpr + k) : 0u;
}

// The word of row `prow` shifted by dx points, from the lane's word w at k
// (the neighbour words come from the adjacent lanes, or are loaded by the
// first and the last lane). Every lane of the warp must take part.
__device__ __forceinline__ uint32_t pshift(const uint32_t* m, int64_t prow, int k, int wpr, bool ok, uint32_t w,
                                           int dx)
{
    const int lane = threadIdx.x & 31;
    uint32_t wl = __shfl_up_sync(kFull, w, 1), wr = __shfl_down_sync(kFull, w, 1);
    if (lane == 0) wl = pword(m, prow, k - 1, wpr, ok);
    if (lane == 31) wr = pword(m, prow, k + 1, wpr, ok);
    if (dx > 0) return __funnelshift_r(w, wr, 2 * dx);
    if (dx < 0) return __funnelshift_l(wl, w, -2 * dx);
    return w;
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

// S at every point, Dist1 where S != 0 off B1, and the queries: one warp per
// row, one packed word (16 points) per lane and step.
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
    const int wpr = a.wpr;
    const uint32_t* cm = a.codes;
    const int wstride = gridDim.x * (blockDim.x >> 5);
    const int* tab = RANK == 3 ? c_near.off3 : c_near.off2;
    bool fail = false;
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += wstride) {
        const int z = RANK == 3 ? row / a.ny : 0;
        const int y = row - z * a.ny;
        for (int ks = 0; ks < wpr; ks += 32) {
            const int k = ks + lane;
            const bool in = k < wpr;
            const uint32_t w = pword(cm, row, k, wpr, true);
            const int nv = a.nx - 16 * k;  // fields of this word inside the row
            const uint32_t valid = !in ? 0u : (nv >= 16 ? 0xFFFFFFFFu : (1u << (2 * nv)) - 1u);
            const uint32_t site = field_lsb(w);
            uint32_t need = ~site & 0x55555555u & valid;  // points off B1
            uint32_t s = w - site;                        // B1: the code less one is S_B
            if (__any_sync(kFull, need != 0)) {
                uint32_t res = 0;     // the code of the site each resolved point took
                uint32_t grp[kNearR2 + 1];  // points resolved at squared distance r2
                const uint32_t need0 = need;
                // squared distance 1, in tie order z-, y-, x-, x+, y+, z+
                auto take = [&](uint32_t v) {
                    const uint32_t t = field_lsb(v) & need;
                    res |= v & (t * 3u);
                    need &= ~t;
                };
                const bool zm = RANK == 3 && z > 0, zp = RANK == 3 && z < a.nz - 1;
                const uint32_t wzm = pword(cm, row - a.ny, k, wpr, zm);
                const uint32_t wym = pword(cm, row - 1, k, wpr, y > 0);
                const uint32_t wyp = pword(cm, row + 1, k, wpr, y < a.ny - 1);
                const uint32_t wzp = pword(cm, row + a.ny, k, wpr, zp);
                const uint32_t wxm = pshift(cm, row, k, wpr, true, w, -1);
                const uint32_t wxp = pshift(cm, row, k, wpr, true, w, 1);
                if (RANK == 3) take(wzm);
                take(wym);
                take(wxm);
                take(wxp);
                take(wyp);
                if (RANK == 3) take(wzp);
                grp[1] = need0 & ~need;
#pragma unroll
                for (int r = 2; r <= kNearR2; ++r) grp[r] = 0;
                if (__any_sync(kFull, need != 0)) {
                    // squared distances 2..8: the rest of the table in order
#pragma unroll
                    for (int r = 2; r <= kNearR2; ++r) {
                        const uint32_t before = need;
                        const int e0 = group_begin(RANK == 3, r), e1 = group_begin(RANK == 3, r + 1);
                        for (int e = e0; e < e1; ++e) {
                            const int o = tab[e];
                            const int dx = (int)(int8_t)(o & 0xFF), dy = (int)(int8_t)((o >> 8) & 0xFF);
                            const int dz = (int)(int8_t)((o >> 16) & 0xFF);
                            const bool ok = (unsigned)(y + dy) < (unsigned)a.ny &&
                                            (RANK == 2 || (unsigned)(z + dz) < (unsigned)a.nz);
                            const int64_t prow = (int64_t)row + (int64_t)dz * a.ny + dy;
                            const uint32_t wr = pword(cm, prow, k, wpr, ok);
                            take(pshift(cm, prow, k, wpr, ok, wr, dx));
                        }
                        grp[r] = before & ~need;
                    }
                    fail |= need != 0;
                }
                const uint32_t resolved = need0 & ~need;
                const uint32_t soff = res - resolved;  // the site's code less one: S
                s |= soff;
                uint32_t qm = field_lsb(soff);         // queries: S != 0 off B1
                while (qm) {
                    const int f = __ffs(qm) - 1;
                    qm &= qm - 1;
                    int r2 = 1;
#pragma unroll
                    for (int r = kNearR2; r >= 1; --r)
                        if ((grp[r] >> f) & 1u) r2 = r;
                    const int code = (int)((soff >> f) & 3u);
                    const int p = row * a.nx + 16 * k + (f >> 1);
                    a.dist1[p] = r2;
                    const Query qe{p, (r2 << 2) | code};
                    const int kq = atomicAdd(&qn, 1);
                    if (kq < kQueryCta) {
                        qbuf[kq] = qe;
                    } else {
                        const int g = atomicAdd(a.ctr + kCtrQueries, 1);
                        if (g < a.qcap) a.qlist[g] = qe;
                    }
                }
            }
            if (in) a.spk[(int64_t)row * wpr + k] = s;
        }
    }
    near_flush(a, qbuf, &qn, &qbase, fail);
}

// The byte maps of the separable passes from q and the packed S: the equal-q
// mask with the sign code of S_B (row pass 1's eqm) and S as int8, after the
// local first EDT (when the separable one ran, its passes wrote them). mode
// 1: only when the separable second EDT takes over (the dense flag set);
// mode 2: always (the adjoint reads them).
template <int RANK, bool VEC>
__global__ void __launch_bounds__(256) k_expand(LocalArgs a, int mode)
{
    wait_prior_grid();
    {
        const volatile int* ctr = a.ctr;
        if (ctr[kCtrLocalFail] != 0 || (mode == 1 && ctr[kCtrDense] == 0)) return;
    }
    const int rows = a.nz * a.ny;
    const int wstride = gridDim.x * (blockDim.x >> 5);
    const int lx = 4 * (int)(threadIdx.x & 31);
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += wstride) {
        const int z = RANK == 3 ? row / a.ny : 0;
        const int y = row - z * a.ny;
        const int64_t rbase = (int64_t)row * a.nx;
        for (int x0 = lx; x0 - lx < a.nx; x0 += 128) {
            SegQ b;
            load_segment<RANK, VEC>(a, row, z, y, x0, b);
            unsigned b1, sg;
            uint32_t em;
            step_a<RANK, true>(a, z, y, x0, b, b1, sg, em);
            const uint32_t sw = x0 < 16 * a.wpr ? __ldg(a.spk + (int64_t)row * a.wpr + (x0 >> 4)) >> (2 * (x0 & 15)) : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (x0 + j >= a.nx) continue;
                const unsigned c = (sw >> (2 * j)) & 3u;
                a.eqm[rbase + x0 + j] = (uint8_t)(em >> (8 * j));
                a.s[rbase + x0 + j] = (int8_t)(c == 1u ? 1 : (c == 2u ? -1 : 0));
            }
        }
    }
}

// The packed S from the int8 S map of the separable first EDT (gated: when
// the local first EDT fell short; else always).
__global__ void __launch_bounds__(256) k_pack_s(LocalArgs a, int gated)
{
    wait_prior_grid();
    if (gated && *static_cast<const volatile int*>(a.ctr + kCtrLocalFail) == 0) return;
    const int64_t words = (int64_t)a.nz * a.ny * a.wpr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) {
        const int64_t row = i / a.wpr;
        const int x0 = 16 * (int)(i - row * a.wpr);
        const int8_t* sr = a.s + row * a.nx;
        uint32_t w = 0;
        for (int j = 0; j < 16 && x0 + j < a.nx; ++j) {
            const int v = sr[x0 + j];
            w |= (v > 0 ? 1u : (v < 0 ? 2u : 0u)) << (2 * j);
        }
        a.spk[i] = w;
    }
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
    auto run = [&](auto kern) { return launch_chained(kern, dim3(one_wave(kern)), dim3(256), 0, st, a); };
    return a.rank == 3 ? run(k_near<3>) : run(k_near<2>);
}

cudaError_t launch_local_expand(const LocalArgs& a, int mode, cudaStream_t st)
{
    auto run = [&](auto kern) {
        return launch_chained(kern, dim3(one_wave(kern)), dim3(256), 0, st, a, mode);
    };
    if (a.rank == 3) return a.vec ? run(k_expand<3, true>) : run(k_expand<3, false>);
    return a.vec ? run(k_expand<2, true>) : run(k_expand<2, false>);
}

cudaError_t launch_local_pack_s(const LocalArgs& a, bool gated, cudaStream_t st)
{
    return launch_chained(k_pack_s, dim3(one_wave(k_pack_s)), dim3(256), 0, st, a, gated ? 1 : 0);
}

}  // namespace qai
