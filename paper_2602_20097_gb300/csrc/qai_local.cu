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
// A point with no B1 point within that ball (or, in 2-D, a warp whose words
// needed the search past squared distance 1 more often than one in 16) sets
// kCtrLocalFail and ends that warp's searches past squared distance 1; the separable
// first EDT (row pass 1, column passes 1) then runs and rewrites all of it,
// and k_pack_s packs its S map for the route. k_expand writes the byte maps
// (equal-q mask, S) that the separable second EDT and the adjoint read.
#include <algorithm>

#include <cuda.h>

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
#define QAI_DETECT_MINB 4
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

// The q values one lane needs for its four points x0 .. x0 + 3 of a row:
// the row, its four neighbour rows (0 where a row does not exist) and the
// values left and right of the four.
struct Quad {
    int c[4], yl[4], yr[4], zl[4], zr[4];
    int xm, xp;
};

// (a ^ c) | (b ^ c) and a | b | c as single three-input logic operations.
template <unsigned LUT>
__device__ __forceinline__ unsigned lop3(unsigned a, unsigned b, unsigned c)
{
    unsigned d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}
constexpr unsigned kLutXorOr = 0x7E;  // (a ^ c) | (b ^ c)
constexpr unsigned kLutOr3 = 0xFE;    // a | b | c

constexpr unsigned kLutXorOrC = 0xBE;  // (a ^ b) | c

// The fast path of step A covers fields whose indices all satisfy
// |q| < 2^26: then every difference and every sum of six differences is
// exact in 32 bits. Each lane checks its own four values (every value of the
// field is some lane's own); a value outside the range sets kCtrWide, and an
// exact pass then redoes step A over the whole field.
constexpr unsigned kNarrowBias = 1u << 26;
__device__ __forceinline__ bool quad_narrow(const Quad& Q)
{
    const unsigned acc = lop3<kLutOr3>((unsigned)Q.c[0] + kNarrowBias, (unsigned)Q.c[1] + kNarrowBias,
                                       ((unsigned)Q.c[2] + kNarrowBias) | ((unsigned)Q.c[3] + kNarrowBias));
    return acc < 2u * kNarrowBias;
}

// Step A (Algorithm 2) for the lane's four points, the sign rule SUM and
// every index in the fast-path range (see quad_narrow). code: 1 in the 2-bit
// field of each B1 point (interior, some axis neighbour differs); sg: the
// sign code of S_B per point (0 off B1 and where the fast-varying test zeroes
// it); ne: per 2-bit field, q != q[x + 1] (low bit) and q != q[y + 1] (high
// bit); nz: q != q[z + 1] (low bit). The ne bits of a missing neighbour are
// not defined (their readers only ask about interior points). Every lane of
// the warp must take part (warp vote).
template <int RANK>
__device__ __forceinline__ void step_a_fast(const MethodArgs& m, bool row_inner, int x0, int nx, const Quad& Q,
                                            unsigned& code, unsigned& sg, unsigned& ne, unsigned& nz)
{
    const int *c = Q.c, *yl = Q.yl, *yr = Q.yr, *zl = Q.zl, *zr = Q.zr;
    const unsigned thm1 = (unsigned)m.grad_threshold - 1u, lim = 2u * thm1;
    code = 0;
    sg = 0;
    ne = 0;
    nz = 0;
    unsigned u[4], ukeep = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned q0 = (unsigned)c[j];
        const unsigned l = (unsigned)(j == 0 ? Q.xm : c[j - 1]);
        const unsigned r = (unsigned)(j == 3 ? Q.xp : c[j + 1]);
        const unsigned tx = r ^ q0, ty = (unsigned)yr[j] ^ q0;
        unsigned d, uz = 0u;
        if (RANK == 3) {
            const unsigned tz = (unsigned)zr[j] ^ q0;
            d = lop3<kLutXorOrC>((unsigned)zl[j], q0, lop3<kLutOr3>(tx, ty, tz)) |
                lop3<kLutXorOr>(l, (unsigned)yl[j], q0);
            uz = (unsigned)zr[j] - (unsigned)zl[j] + thm1;
            nz += min(tz, 1u) << (2 * j);
        } else {
            d = (tx | ty) | lop3<kLutXorOr>(l, (unsigned)yl[j], q0);
        }
        ne += (min(tx, 1u) + 2u * min(ty, 1u)) << (2 * j);
        // the largest of (q[+1] - q[-1] + thm1) over the axes, unsigned:
        // above 2 thm1 exactly when some axis is fast-varying
        u[j] = __vimax3_u32(r - l + thm1, (unsigned)yr[j] - (unsigned)yl[j] + thm1, uz);
        const unsigned b = min(d, 1u);
        code += b << (2 * j);
        ukeep = min(ukeep, u[j] | (b - 1u));  // only B1 points can keep a sign
    }
    if (!row_inner) {  // warp-uniform: off the interior nothing is on B1
        code = 0;
        return;
    }
    // interior along x: x in [1, nx - 2]
    unsigned inner = x0 == 0 ? 0xFCu : 0xFFu;
    const int rem = nx - 1 - x0;  // points x0 .. x0 + rem - 1 are below nx - 1
    if (rem < 4) inner &= rem > 0 ? (1u << (2 * rem)) - 1u : 0u;
    code &= inner;
    if (__any_sync(kFull, ukeep <= lim)) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!((code >> (2 * j)) & 1u) || u[j] > lim) continue;
            const int l = j == 0 ? Q.xm : c[j - 1];
            const int r = j == 3 ? Q.xp : c[j + 1];
            int sum = l + r + yl[j] + yr[j] - 2 * RANK * c[j];
            if (RANK == 3) sum += zl[j] + zr[j];
            sg |= (sum > 0 ? 1u : (sum < 0 ? 2u : 0u)) << (2 * j);
        }
    }
}

// Step A for the lane's four points by the general form (any indices, both
// sign rules; 64-bit sums): code and sg as step_a_fast, the differ bits ne
// and nz, and em, the equal-q mask byte per point (bits z-, z+, y-, y+, x-,
// x+; 0x3F off the interior) with the sign code in bits 6-7: the byte map of
// the separable passes.
template <int RANK>
__device__ __forceinline__ void step_a_exact(const MethodArgs& m, bool row_inner, int x0, int nx, const Quad& Q,
                                             unsigned& code, unsigned& sg, unsigned& ne, unsigned& nz, uint32_t& em)
{
    code = 0;
    sg = 0;
    ne = 0;
    nz = 0;
    em = 0x3F3F3F3Fu;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int r = j == 3 ? Q.xp : Q.c[j + 1];
        ne |= ((Q.c[j] != r ? 1u : 0u) | (Q.c[j] != Q.yr[j] ? 2u : 0u)) << (2 * j);
        if (RANK == 3) nz |= (Q.c[j] != Q.zr[j] ? 1u : 0u) << (2 * j);
    }
    if (!row_inner) return;
    em = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool in = x0 + j >= 1 && x0 + j <= nx - 2;
        const int l = j == 0 ? Q.xm : Q.c[j - 1];
        const int r = j == 3 ? Q.xp : Q.c[j + 1];
        unsigned mk;
        bool site;
        int cd;
        detect_point<RANK, true>(Q.c[j], Q.zl[j], Q.zr[j], Q.yl[j], Q.yr[j], l, r, in, m, mk, site, cd);
        code |= site ? 1u << (2 * j) : 0u;
        sg |= (unsigned)cd << (2 * j);  // 0 off the interior
        em |= ((in ? mk : 0x3Fu) | (unsigned)cd << 6) << (8 * j);
    }
}

// The outputs of step A for the lane's four points of row `row`: D''
// wherever Dist2 does not matter (D' + S_B eta eps on B1, D' elsewhere: the
// expressions of compensate(), with C = +0 the fma is the product), the code
// byte and the differ bytes (up to the row's last packed word).
// The B1 points with S != 0 of a CTA, collected in shared memory and
// appended to the signed list with one atomic when the CTA ends.
constexpr int kSignedCta = 1024, kSignedTma = 512;
struct SignedBuf {
    int32_t* e;
    int* n;
    int cap;
};

template <int RANK, bool VEC>
__device__ __forceinline__ void store_step_a(const LocalArgs& a, int row, int x0, const Quad& Q, unsigned code,
                                             unsigned sg, unsigned ne, unsigned nz, const SignedBuf& sb)
{
    const int nx = a.nx;
    float* orow = a.out + (int64_t)row * nx;
    float o[4];
    if (__any_sync(kFull, sg != 0)) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned cd = (sg >> (2 * j)) & 3u;
            const float cc = (cd == 1u ? 1.0f : (cd == 2u ? -1.0f : 0.0f)) * a.m.eta_eb;
            o[j] = a.m.output_c ? cc : fmaf((float)Q.c[j], a.m.two_eb, cc);
            // past the CTA's buffer the list is incomplete whatever the count
            if (cd && *static_cast<volatile int*>(sb.n) <= sb.cap) {
                const int k = atomicAdd(sb.n, 1);
                if (k < sb.cap) sb.e[k] = row * nx + x0 + j;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = a.m.output_c ? 0.0f : (float)Q.c[j] * a.m.two_eb;
    }
    if (VEC) {
        if (x0 < nx) *reinterpret_cast<float4*>(orow + x0) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (x0 + j < nx) orow[x0 + j] = o[j];
    }
    if (x0 < 16 * a.wpr) {
        const int64_t b = (int64_t)row * 4 * a.wpr + (x0 >> 2);
        reinterpret_cast<uint8_t*>(a.codes)[b] = (uint8_t)(code + sg);
        reinterpret_cast<uint8_t*>(a.nexy)[b] = (uint8_t)ne;
        if (RANK == 3) reinterpret_cast<uint8_t*>(a.nez)[b] = (uint8_t)nz;
    }
}

// The Quad of the lane's four points of row `row` from global memory: one
// 128-bit load per row when VEC (x0 and the rows 16-byte aligned), the x
// neighbours from the adjacent lanes (the first and the last lane load
// theirs). Every lane of the warp must take part.
template <int RANK, bool VEC>
__device__ __forceinline__ void load_quad(const LocalArgs& a, int row, int z, int y, int x0, Quad& Q)
{
    const int lane = threadIdx.x & 31;
    const int nx = a.nx;
    const int32_t* qr = a.q + (int64_t)row * nx;
    const int64_t plane = (int64_t)a.ny * nx;
    load4_i32(qr, x0, nx, VEC, Q.c);
#pragma unroll
    for (int j = 0; j < 4; ++j) Q.yl[j] = Q.yr[j] = Q.zl[j] = Q.zr[j] = 0;
    if (y >= 1) load4_i32(qr - nx, x0, nx, VEC, Q.yl);
    if (y + 1 < a.ny) load4_i32(qr + nx, x0, nx, VEC, Q.yr);
    if (RANK == 3) {
        if (z >= 1) load4_i32(qr - plane, x0, nx, VEC, Q.zl);
        if (z + 1 < a.nz) load4_i32(qr + plane, x0, nx, VEC, Q.zr);
    }
    Q.xm = __shfl_up_sync(kFull, Q.c[3], 1);
    Q.xp = __shfl_down_sync(kFull, Q.c[0], 1);
    if (lane == 0) Q.xm = x0 > 0 ? __ldg(qr + x0 - 1) : 0;
    if (lane == 31) Q.xp = x0 + 4 < nx ? __ldg(qr + x0 + 4) : 0;
}

// Step A, one warp per row, 128 points per step (the form for 2-D fields, for
// rows that are not 16-byte multiples and for the exact pass). mode 0: the
// fast path, flagging a field with an index outside its range; 1: the exact
// form; 2: the exact form, only when the flag is set.
// The CTA's signed points to the list (one atomic); a CTA with more than its
// buffer holds marks the list incomplete.
__device__ __forceinline__ void flush_signed(const LocalArgs& a, const SignedBuf& sb, int* base)
{
    __syncthreads();
    const int n = *sb.n;
    if (threadIdx.x == 0) {
        *base = -1;
        if (n > sb.cap) *static_cast<volatile int*>(a.ctr + kCtrSignedOver) = 1;
        else if (n > 0) *base = atomicAdd(a.ctr + kCtrSigned, n);
    }
    __syncthreads();
    if (*base >= 0)
        for (int i = threadIdx.x; i < n && *base + i < a.scap; i += blockDim.x) a.slist[*base + i] = sb.e[i];
}

template <int RANK, bool VEC>
__device__ __forceinline__ void k_detect_body(const LocalArgs& a, int mode, const int bx, const int gx)
{
    __shared__ int32_t sbuf[kSignedCta];
    __shared__ int sn, sbase;
    wait_prior_grid();
    if (mode == 2 && *static_cast<const volatile int*>(a.ctr + kCtrWide) == 0) return;
    if (threadIdx.x == 0) sn = 0;
    __syncthreads();
    const SignedBuf sb{sbuf, &sn, kSignedCta};
    const int rows = a.nz * a.ny;
    const int wstride = gx * (blockDim.x >> 5);
    const int lx = 4 * (int)(threadIdx.x & 31);
    bool wide = false;
    for (int row = bx * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += wstride) {
        const int z = RANK == 3 ? row / a.ny : 0;
        const int y = row - z * a.ny;
        const bool row_inner = y >= 1 && y <= a.ny - 2 && (RANK == 2 || (z >= 1 && z <= a.nz - 2));
        for (int x0 = lx; x0 - lx < a.nx; x0 += 128) {
            Quad Q;
            load_quad<RANK, VEC>(a, row, z, y, x0, Q);
            unsigned code, sg, ne, nz;
            if (mode == 0) {
                wide |= !quad_narrow(Q);
                step_a_fast<RANK>(a.m, row_inner, x0, a.nx, Q, code, sg, ne, nz);
            } else {
                uint32_t em;
                step_a_exact<RANK>(a.m, row_inner, x0, a.nx, Q, code, sg, ne, nz, em);
            }
            store_step_a<RANK, VEC>(a, row, x0, Q, code, sg, ne, nz, sb);
        }
    }
    if (__any_sync(kFull, wide) && (threadIdx.x & 31) == 0) *static_cast<volatile int*>(a.ctr + kCtrWide) = 1;
    if (mode != 2) {
        flush_signed(a, sb, &sbase);
    } else {
        // the exact pass: the fast pass's list may be wrong; the count stands
        // apart and the list is marked incomplete
        __syncthreads();
        if (threadIdx.x == 0) {
            if (sn) atomicAdd(a.ctr + kCtrSignedExact, sn);
            if (bx == 0) *static_cast<volatile int*>(a.ctr + kCtrSignedOver) = 1;
        }
    }
}

template <int RANK, bool VEC>
__global__ void __launch_bounds__(256, QAI_DETECT_MINB) k_detect(LocalArgs a, int mode)
{
    k_detect_body<RANK, VEC>(a, mode, blockIdx.x, gridDim.x);
}


// ---- step A for 3-D fields on tiles staged by the tensor memory accelerator
//
// A CTA walks runs of consecutive z-planes of (x, y) tiles of kTX x kTY
// points. Each plane of a tile, with a one-point halo in y and a four-point
// halo in x (the copy starts on a 16-byte boundary), comes into shared memory
// as one TMA box copy (points outside the field read 0); a ring of four
// plane buffers holds planes z - 1, z, z + 1 while z + 2 is in flight, so
// every q value crosses from L2 into the SM once per tile. The steps of all
// tiles (tile-major, z fastest) are split evenly over the CTAs.
constexpr int kTX = 128, kTY = 32;
constexpr int kBoxX = kTX + 8, kBoxY = kTY + 2;
constexpr int kPlaneInts = kBoxX * kBoxY;
constexpr int kSlotInts = (kPlaneInts + 31) / 32 * 32;  // 128-byte multiples
constexpr int kSlots = 4;
constexpr size_t kTmaSmem = (size_t)kSlots * kSlotInts * 4 + kSlots * 8;
static_assert((kBoxX * 4) % 16 == 0, "TMA box rows are 16-byte multiples");
static_assert(kTY % 8 == 0, "eight warps share a tile's rows");
constexpr unsigned kWaitLimit = 1u << 22;  // polls of a plane's barrier before the kernel gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Plane z of tile (x0t, y0t) into the ring slot of z, completing on the
// slot's barrier (one thread).
__device__ __forceinline__ void tma_plane(const CUtensorMap* tm, int* slot, uint64_t* bar, int x0t, int y0t, int z)
{
    const uint32_t b = smem_u32(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"((uint32_t)(kPlaneInts * 4))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(slot)), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x0t - 4), "r"(y0t - 1), "r"(z), "r"(b)
        : "memory");
}

// Waits (bounded) for the current phase of a slot's barrier; false if the
// limit ran out.
__device__ __forceinline__ bool wait_plane(uint64_t* bar, uint32_t parity)
{
    const uint32_t b = smem_u32(bar);
    for (unsigned i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(b), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(256, 3) k_detect_tma(LocalArgs a, const __grid_constant__ CUtensorMap tm,
                                                      int tiles_x, int zb, int zn)
{
    extern __shared__ __align__(128) int sbuf[];  // the plane ring, then the slots' barriers
    uint64_t* bars = reinterpret_cast<uint64_t*>(sbuf + kSlots * kSlotInts);
    __shared__ int32_t signed_buf[kSignedTma];
    __shared__ int sn, sbase;
    const SignedBuf sb{signed_buf, &sn, kSignedTma};
    wait_prior_grid();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sn = 0;
    }
    __syncthreads();
    uint32_t parity = 0;  // bit s: the phase parity slot s completes next
    bool timed_out = false, wide = false;
    // planes zb .. zb + zn - 1 of every tile (the whole field, or one slab)
    const int nz = a.nz;
    const int64_t steps = (int64_t)tiles_x * ((a.ny + kTY - 1) / kTY) * zn;
    const int64_t s0 = steps * blockIdx.x / gridDim.x, s1 = steps * (blockIdx.x + 1) / gridDim.x;
    auto slot_of = [](int z) { return ((z % kSlots) + kSlots) % kSlots; };
    for (int64_t s = s0; s < s1;) {
        // a run of planes z0 .. z1 - 1 of one tile
        const int tile = (int)(s / zn);
        const int z0 = zb + (int)(s - (int64_t)tile * zn);
        const int z1 = (int)min((int64_t)zb + zn, (int64_t)z0 + (s1 - s));
        const int x0t = (tile % tiles_x) * kTX, y0t = (tile / tiles_x) * kTY;
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int p = z0 - 1; p <= min(z0 + 2, z1); ++p)
                tma_plane(&tm, sbuf + slot_of(p) * kSlotInts, &bars[slot_of(p)], x0t, y0t, p);
        }
        for (int z = z0; z < z1; ++z) {
            for (int p = (z == z0 ? z0 - 1 : z + 1); p <= z + 1; ++p) {
                const int sl = slot_of(p);
                if (!wait_plane(&bars[sl], (parity >> sl) & 1u)) timed_out = true;
                parity ^= 1u << sl;
            }
            const int* P0 = sbuf + slot_of(z) * kSlotInts;
            const int* Pm = sbuf + slot_of(z - 1) * kSlotInts;
            const int* Pp = sbuf + slot_of(z + 1) * kSlotInts;
            const int x0 = x0t + 4 * lane;
#pragma unroll 1
            for (int r = warp; r < kTY; r += 8) {
                const int y = y0t + r;
                if (y >= a.ny) break;  // warp-uniform
                const int o = (r + 1) * kBoxX + 4 + 4 * lane;
                Quad Q;
                auto ld4s = [](const int* p, int v[4]) {
                    const int4 t = *reinterpret_cast<const int4*>(p);
                    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
                };
                ld4s(P0 + o, Q.c);
                ld4s(P0 + o - kBoxX, Q.yl);
                ld4s(P0 + o + kBoxX, Q.yr);
                ld4s(Pm + o, Q.zl);
                ld4s(Pp + o, Q.zr);
                Q.xm = P0[o - 1];
                Q.xp = P0[o + 4];
                const int row = z * a.ny + y;
                const bool row_inner = y >= 1 && y <= a.ny - 2 && z >= 1 && z <= nz - 2;
                unsigned code, sg, ne, nzb;
                wide |= !quad_narrow(Q);
                step_a_fast<3>(a.m, row_inner, x0, a.nx, Q, code, sg, ne, nzb);
                store_step_a<3, true>(a, row, x0, Q, code, sg, ne, nzb, sb);
            }
            __syncthreads();  // every read of plane z - 1 done: its slot takes z + 3
            if (threadIdx.x == 0 && z + 3 <= z1) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_plane(&tm, sbuf + slot_of(z + 3) * kSlotInts, &bars[slot_of(z + 3)], x0t, y0t, z + 3);
            }
        }
        s += z1 - z0;
    }
    if (timed_out && lane == 0) *static_cast<volatile int*>(a.ctr + kCtrTimeout) = 1;
    if (__any_sync(kFull, wide) && lane == 0) *static_cast<volatile int*>(a.ctr + kCtrWide) = 1;
    flush_signed(a, sb, &sbase);
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
__device__ __forceinline__ void near_flush(const LocalArgs& a, const Query* qbuf, const int* qn, int* qbase)
{
    __syncthreads();
    const int n = min(*qn, kQueryCta);
    if (threadIdx.x == 0) *qbase = n > 0 ? atomicAdd(a.ctr + kCtrQueries, n) : 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n && *qbase + i < a.qcap; i += blockDim.x) a.qlist[*qbase + i] = qbuf[i];
}

// Squared distance from (z, y, x) to the first B1 point among the table
// entries of squared length >= 2 (in table order); 0 if none.
template <int RANK>
__device__ __forceinline__ int deep_r2(const LocalArgs& a, int z, int y, int x)
{
    const int* tab = RANK == 3 ? c_near.off3 : c_near.off2;
    constexpr int n1 = RANK == 3 ? 6 : 4, ntab = RANK == 3 ? kNearN3 : kNearN2;
    for (int e = n1; e < ntab; ++e) {
        const int o = tab[e];
        const int xx = x + (int)(int8_t)(o & 0xFF), yy = y + (int)(int8_t)((o >> 8) & 0xFF);
        const int zz = z + (int)(int8_t)((o >> 16) & 0xFF);
        if ((unsigned)xx >= (unsigned)a.nx || (unsigned)yy >= (unsigned)a.ny || (unsigned)zz >= (unsigned)a.nz) continue;
        const uint32_t w = __ldg(a.codes + ((int64_t)zz * a.ny + yy) * a.wpr + (xx >> 4));
        if ((w >> (2 * (xx & 15))) & 3u) return (int)((unsigned)o >> 24);
    }
    return 0;
}

// S at every point, Dist1 where S != 0 off B1, and the queries. A warp takes
// kNearRows rows of one plane at a time, one packed word (16 points) per
// lane and step, with the words of all the rows it needs loaded up front.
// The six neighbours at squared distance 1 are tested for all words at once;
// a word with a point still unresolved after them is searched by the whole
// warp, 32 table entries at a time (a lane per entry), the first entry in
// table order with a site taking each point.
constexpr int kNearRows = 4;

// DYN (the one-field launch, when near_stride is set): after its first item
// the warp takes the next from a counter in the route words, fetched while it
// works on the current one -- the cost of an item varies with the searches
// it needs, and over many rounds a fixed split leaves a few SMs working long
// after the rest. The t-th item handed out is t * near_stride mod items (a
// stride prime to the count), so that the items in work at one time are
// spread over the field, as the fixed split spreads them. The fixed split
// keeps the eight warps of a CTA on adjacent rows (their shared halo rows hit
// in L1), which wins when each warp has few items; the grouped launch keeps
// it always.
template <int RANK, bool DYN = false>
__device__ __forceinline__ void k_near_body(const LocalArgs& a, const int bx, const int gx)
{
    wait_prior_grid();
    __shared__ Query qbuf[kQueryCta];
    __shared__ int qn, qbase;
    if (threadIdx.x == 0) qn = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wpr = a.wpr;
    const uint32_t* cm = a.codes;
    const int yb = (a.ny + kNearRows - 1) / kNearRows;
    const int items = a.nz * yb;
    const int wstride = gx * (blockDim.x >> 5);
    const int* tab = RANK == 3 ? c_near.off3 : c_near.off2;
    constexpr int n1 = RANK == 3 ? 6 : 4, ntab = RANK == 3 ? kNearN3 : kNearN2;
    // A warp gives up -- sets the flag, after which the separable passes
    // redo every output, and skips its remaining searches past squared
    // distance 1 -- at a point without a site within reach, or (2-D fields,
    // whose separable passes are cheap next to a wide search) when more than
    // one in 16 of the words it has looked at (plus 16) needed such a
    // search. The loop reads no shared state, so nothing stalls the loads it
    // issues up front (warps of a field that fails meet either test soon).
    bool fail = false;  // warp-uniform
    int seen = 0, deep = 0;  // warp-uniform: words looked at, words searched past squared distance 1
    // the first item of every warp is fixed (no burst of atomics at the start)
    constexpr bool dyn = DYN;
    int t = bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
    while (t < items) {
        int next = 0;  // dyn: the warp's next item, fetched ahead
        if (dyn && lane == 0) next = wstride + atomicAdd(a.ctr + kCtrNearItems, 1);
        const int it = dyn ? (int)((int64_t)t * a.near_stride % items) : t;
        const int z = RANK == 3 ? it / yb : 0;
        const int y0 = (it - z * yb) * kNearRows;
        const int row0 = z * a.ny + y0;
        for (int ks = 0; ks < wpr; ks += 32) {
            const int k = ks + lane;
            const bool in = k < wpr;
            // rows y0 - 1 .. y0 + kNearRows of this plane; planes z -+ 1
            uint32_t wy[kNearRows + 2], wzm[kNearRows], wzp[kNearRows];
#pragma unroll
            for (int i = 0; i < kNearRows + 2; ++i) {
                const int y = y0 - 1 + i;
                wy[i] = pword(cm, (int64_t)row0 - 1 + i, k, wpr, y >= 0 && y < a.ny);
            }
#pragma unroll
            for (int i = 0; i < kNearRows; ++i) {
                const bool ok = RANK == 3 && y0 + i < a.ny;
                wzm[i] = pword(cm, (int64_t)row0 + i - a.ny, k, wpr, ok && z > 0);
                wzp[i] = pword(cm, (int64_t)row0 + i + a.ny, k, wpr, ok && z < a.nz - 1);
            }
            const int nv = a.nx - 16 * k;  // fields of this word inside the row
            const uint32_t valid = !in ? 0u : (nv >= 16 ? 0xFFFFFFFFu : (1u << (2 * nv)) - 1u);
#pragma unroll
            for (int i = 0; i < kNearRows; ++i) {
                const int y = y0 + i;
                if (y >= a.ny) break;  // warp-uniform
                const int row = row0 + i;
                const uint32_t w = wy[i + 1];
                if (RANK == 2) seen += min(32, wpr - ks);
                const uint32_t site = field_lsb(w);
                uint32_t need = ~site & 0x55555555u & valid;  // points off B1
                uint32_t s = w - site;                        // B1: the code less one is S_B
                if (__any_sync(kFull, need != 0)) {
                    uint32_t res = 0;  // the code of the site each resolved point took
                    const uint32_t need0 = need;
                    // squared distance 1, in tie order z-, y-, x-, x+, y+, z+
                    auto take = [&](uint32_t v) {
                        const uint32_t t = field_lsb(v) & need;
                        res |= v & (t * 3u);
                        need &= ~t;
                    };
                    const uint32_t wxm = pshift(cm, row, k, wpr, true, w, -1);
                    const uint32_t wxp = pshift(cm, row, k, wpr, true, w, 1);
                    const uint32_t all6 = (RANK == 3 ? wzm[i] | wzp[i] : 0u) | wy[i] | wy[i + 2] | wxm | wxp;
                    if (__any_sync(kFull, (need & (all6 >> 1)) != 0)) {
                        if (RANK == 3) take(wzm[i]);
                        take(wy[i]);
                        take(wxm);
                        take(wxp);
                        take(wy[i + 2]);
                        if (RANK == 3) take(wzp[i]);
                    } else {
                        // no point off B1 has a signed neighbour at squared
                        // distance 1 (a code >= 2): whichever of them comes
                        // first carries S_B = 0 (code 1)
                        const uint32_t t = field_lsb(all6) & need;
                        res = t;
                        need &= ~t;
                    }
                    const uint32_t at1 = need0 & ~need;  // resolved at squared distance 1
                    // squared distances 2..8: the words with a point left, one
                    // at a time, searched by the warp -- within a budget of
                    // such words for the field (one in 16), past which the
                    // separable passes are the cheaper first EDT
                    unsigned needy = __ballot_sync(kFull, need != 0);
                    if (needy) {
                        if (RANK == 2) {
                            deep += __popc(needy);
                            if (!fail && 16 * deep > seen + 256) {
                                if (lane == 0) *static_cast<volatile int*>(a.ctr + kCtrLocalFail) = 1;
                                fail = true;
                            }
                        }
                        if (fail) needy = 0;
                    }
                    for (; needy; needy &= needy - 1) {
                        const int src = __ffs(needy) - 1;
                        const int kk = __shfl_sync(kFull, k, src);
                        uint32_t nd = __shfl_sync(kFull, need, src);
                        uint32_t rs = 0;
                        for (int base = n1; base < ntab && nd; base += 32) {
                            const int e = base + lane;
                            uint32_t t = 0, v = 0;
                            if (e < ntab) {
                                const int o = tab[e];
                                const int dx = (int)(int8_t)(o & 0xFF), dy = (int)(int8_t)((o >> 8) & 0xFF);
                                const int dz = (int)(int8_t)((o >> 16) & 0xFF);
                                const bool ok = (unsigned)(y + dy) < (unsigned)a.ny &&
                                                (RANK == 2 || (unsigned)(z + dz) < (unsigned)a.nz);
                                const int64_t prow = (int64_t)row + (int64_t)dz * a.ny + dy;
                                const uint32_t w0 = pword(cm, prow, kk, wpr, ok);
                                const uint32_t wn = pword(cm, prow, dx > 0 ? kk + 1 : kk - 1, wpr, ok && dx != 0);
                                v = dx > 0 ? __funnelshift_r(w0, wn, 2 * dx)
                                           : (dx < 0 ? __funnelshift_l(wn, w0, -2 * dx) : w0);
                                t = field_lsb(v) & nd;
                            }
                            // each point goes to the first entry (lowest lane) with a site
                            uint32_t incl = t;
#pragma unroll
                            for (int d = 1; d < 32; d <<= 1) {
                                const uint32_t x = __shfl_up_sync(kFull, incl, d);
                                if (lane >= d) incl |= x;
                            }
                            uint32_t excl = __shfl_up_sync(kFull, incl, 1);
                            if (lane == 0) excl = 0;
                            rs |= v & ((t & ~excl) * 3u);
                            nd &= ~__shfl_sync(kFull, incl, 31);
                        }
                        rs = __reduce_or_sync(kFull, rs);
                        if (lane == src) {
                            res |= rs;
                            need = nd;
                        }
                    }
                    if (!fail && __any_sync(kFull, need != 0)) {
                        if (lane == 0) *static_cast<volatile int*>(a.ctr + kCtrLocalFail) = 1;
                        fail = true;
                    }
                    const uint32_t resolved = need0 & ~need;
                    const uint32_t soff = res - resolved;  // the site's code less one: S
                    s |= soff;
                    // queries: S != 0 off B1 (none once a warp of a 2-D
                    // field gave up: the separable passes then redo Dist1
                    // and the list)
                    uint32_t qm = RANK == 2 && fail ? 0u : field_lsb(soff);
                    while (qm) {
                        const int f = __ffs(qm) - 1;
                        qm &= qm - 1;
                        const int x = 16 * k + (f >> 1);
                        const int r2 = (at1 >> f) & 1u ? 1 : deep_r2<RANK>(a, z, y, x);
                        const int code = (int)((soff >> f) & 3u);
                        const int p = row * a.nx + x;
                        a.dist1[p] = r2;
                        const Query qe{p, (r2 << 2) | code};
                        const int kq = atomicAdd(&qn, 1);
                        if (kq < kQueryCta) {
                            qbuf[kq] = qe;
                        } else if (*static_cast<const volatile int*>(a.ctr + kCtrQueries) <= a.qcap) {
                            // past the list's capacity the route hands over: no more atomics
                            const int g = atomicAdd(a.ctr + kCtrQueries, 1);
                            if (g < a.qcap) a.qlist[g] = qe;
                        }
                    }
                }
                if (in) a.spk[(int64_t)row * wpr + k] = s;
            }
        }
        t = dyn ? __shfl_sync(kFull, next, 0) : t + wstride;
    }
    near_flush(a, qbuf, &qn, &qbase);
}

template <int RANK, bool DYN>
__global__ void __launch_bounds__(256, QAI_NEAR_MINB) k_near(LocalArgs a)
{
    k_near_body<RANK, DYN>(a, blockIdx.x, gridDim.x);
}


// The byte maps of the separable passes from q and the packed S: the equal-q
// mask with the sign code of S_B (row pass 1's eqm) and S as int8, after the
// local first EDT (when the separable one ran, its passes wrote them). mode
// 1: only when the separable second EDT takes over (the dense flag set);
// mode 2: always (the adjoint reads them).
template <int RANK, bool VEC>
__device__ __forceinline__ void k_expand_body(const LocalArgs& a, int mode, const int bx, const int gx)
{
    wait_prior_grid();
    {
        const volatile int* ctr = a.ctr;
        if (ctr[kCtrLocalFail] != 0 || (mode == 1 && ctr[kCtrDense] == 0)) return;
    }
    const int rows = a.nz * a.ny;
    const int wstride = gx * (blockDim.x >> 5);
    const int lx = 4 * (int)(threadIdx.x & 31);
    for (int row = bx * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += wstride) {
        const int z = RANK == 3 ? row / a.ny : 0;
        const int y = row - z * a.ny;
        const int64_t rbase = (int64_t)row * a.nx;
        const bool row_inner = y >= 1 && y <= a.ny - 2 && (RANK == 2 || (z >= 1 && z <= a.nz - 2));
        for (int x0 = lx; x0 - lx < a.nx; x0 += 128) {
            Quad Q;
            load_quad<RANK, VEC>(a, row, z, y, x0, Q);
            unsigned code, sg, ne, nz;
            uint32_t em;
            step_a_exact<RANK>(a.m, row_inner, x0, a.nx, Q, code, sg, ne, nz, em);
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

template <int RANK, bool VEC>
__global__ void __launch_bounds__(256) k_expand(LocalArgs a, int mode)
{
    k_expand_body<RANK, VEC>(a, mode, blockIdx.x, gridDim.x);
}


// The packed S from the int8 S map of the separable first EDT (gated: when
// the local first EDT fell short; else always).
__device__ __forceinline__ void k_pack_s_body(const LocalArgs& a, int gated, const int bx, const int gx)
{
    wait_prior_grid();
    if (gated && *static_cast<const volatile int*>(a.ctr + kCtrLocalFail) == 0) return;
    const int64_t words = (int64_t)a.nz * a.ny * a.wpr;
    const int64_t stride = (int64_t)gx * blockDim.x;
    for (int64_t i = (int64_t)bx * blockDim.x + threadIdx.x; i < words; i += stride) {
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

__global__ void __launch_bounds__(256) k_pack_s(LocalArgs a, int gated)
{
    k_pack_s_body(a, gated, blockIdx.x, gridDim.x);
}


// The host-memory pipeline's last step: step A's slabs went to the host as
// soon as they were written; the outputs that changed after it go straight
// into the caller's mapped host buffer -- the queries' outputs (the routes of
// the second EDT write nothing else), or every output when a pass that
// rewrites more ran (the exact step A, the separable first EDT, the dense
// second EDT) or a bounded wait ran out. vec: 16-byte aligned, N a multiple
// of 4.
__global__ void __launch_bounds__(256) k_host_fixup(LocalArgs a, float* h_out, int vec)
{
    wait_prior_grid();
    const volatile int* ctr = a.ctr;
    const bool all = ctr[kCtrWide] || ctr[kCtrLocalFail] || ctr[kCtrDense] || ctr[kCtrTimeout];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (all) {
        const int64_t N = (int64_t)a.nz * a.ny * a.nx;
        if (vec) {
            for (int64_t i = t0; i < N / 4; i += stride)
                reinterpret_cast<float4*>(h_out)[i] = __ldg(reinterpret_cast<const float4*>(a.out) + i);
        } else {
            for (int64_t i = t0; i < N; i += stride) h_out[i] = a.out[i];
        }
        return;
    }
    const int nq = min((int)ctr[kCtrQueries], a.qcap);
    for (int64_t i = t0; i < nq; i += stride) {
        const int p = a.qlist[i].idx;
        h_out[p] = a.out[p];
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

namespace {
// cuTensorMapEncodeTiled, found once through the runtime (no link-time
// dependency on the driver library).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled()
{
    static EncodeTiled fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

// The tensor map of q as an (nx, ny, nz) int32 array with kBoxX x kBoxY x 1
// boxes (points outside the array read 0); false if it cannot be made.
bool q_tensor_map(const LocalArgs& a, CUtensorMap* tm)
{
    EncodeTiled enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny, (cuuint64_t)a.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)a.nx * 4, (cuuint64_t)a.nx * a.ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kBoxX, (cuuint32_t)kBoxY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_INT32, 3, const_cast<int32_t*>(a.q), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

// The fast path of step A: the tiled form for 3-D fields of 16-byte rows, the
// row form otherwise.
static bool tma_form(const LocalArgs& a) { return a.rank == 3 && a.vec && encode_tiled() != nullptr; }

// The tiled fast path over planes zb .. zb + zn - 1.
static cudaError_t fast_detect_planes(const LocalArgs& a, int zb, int zn, cudaStream_t st)
{
    CUtensorMap tm;
    if (!q_tensor_map(a, &tm)) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_detect_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int dev = 0, sms = 152, per = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_detect_tma, 256, kTmaSmem) != cudaSuccess || per < 1)
        per = 1;
    const int tiles_x = (a.nx + kTX - 1) / kTX, tiles_y = (a.ny + kTY - 1) / kTY;
    const int64_t steps = (int64_t)tiles_x * tiles_y * zn;
    const int grid = (int)std::min<int64_t>(steps, (int64_t)sms * per);
    return launch_chained(k_detect_tma, dim3(grid), dim3(256), kTmaSmem, st, a, tm, tiles_x, zb, zn);
}

static cudaError_t fast_detect(const LocalArgs& a, cudaStream_t st)
{
    auto run = [&](auto kern) {
        return launch_chained(kern, dim3(one_wave(kern, QAI_DETECT_WAVES)), dim3(256), 0, st, a, 0);
    };
    if (tma_form(a)) return fast_detect_planes(a, 0, a.nz, st);
    if (a.rank == 3) return a.vec ? run(k_detect<3, true>) : run(k_detect<3, false>);
    return a.vec ? run(k_detect<2, true>) : run(k_detect<2, false>);
}

bool local_detect_slabs(const LocalArgs& a) { return a.m.sign_rule == 0 && tma_form(a); }

cudaError_t launch_local_detect_slab(const LocalArgs& a, int zb, int zn, cudaStream_t st)
{
    return fast_detect_planes(a, zb, zn, st);
}

cudaError_t launch_local_detect_exact(const LocalArgs& a, cudaStream_t st)
{
    auto run = [&](auto kern) {
        return launch_chained(kern, dim3(one_wave(kern, QAI_DETECT_WAVES)), dim3(256), 0, st, a, 2);
    };
    if (a.rank == 3) return a.vec ? run(k_detect<3, true>) : run(k_detect<3, false>);
    return a.vec ? run(k_detect<2, true>) : run(k_detect<2, false>);
}

cudaError_t launch_local_detect(const LocalArgs& a, cudaStream_t st)
{
    // the exact pass: after the fast path, gated on its flag; alone under the
    // sign rule FIRST (no fast path)
    auto exact = [&](int mode) {
        auto run = [&](auto kern) {
            return launch_chained(kern, dim3(one_wave(kern, QAI_DETECT_WAVES)), dim3(256), 0, st, a, mode);
        };
        if (a.rank == 3) return a.vec ? run(k_detect<3, true>) : run(k_detect<3, false>);
        return a.vec ? run(k_detect<2, true>) : run(k_detect<2, false>);
    };
    if (a.m.sign_rule != 0) return exact(1);
    cudaError_t e = fast_detect(a, st);
    return e != cudaSuccess ? e : exact(2);
}

cudaError_t launch_local_near(const LocalArgs& a_in, cudaStream_t st)
{
    LocalArgs a = a_in;
    // items handed out from the counter when every warp has eight or more
    // (measured: 13 a warp on 512^3 gains 13 %, 6 on 98 x 1200^2 loses 14 %),
    // in the order of a stride prime to the count near its golden section;
    // the fixed split is a kernel of its own (the counter's code in the
    // kernel slows the fixed split by as much)
    const int64_t items = (int64_t)a.nz * ((a.ny + kNearRows - 1) / kNearRows);
    const int grid = a.rank == 3 ? one_wave(k_near<3, false>) : one_wave(k_near<2, false>);
    a.near_stride = 0;
    if (items >= (int64_t)8 * grid * 8) {
        int64_t sd = std::max<int64_t>(1, (int64_t)(0.6180339887 * (double)items)) | 1;
        auto gcd = [](int64_t u, int64_t v) { while (v) { const int64_t r = u % v; u = v; v = r; } return u; };
        while (gcd(sd, items) != 1) sd += 2;
        a.near_stride = (int)(sd % items);
    }
    auto run = [&](auto kern) { return launch_chained(kern, dim3(one_wave(kern)), dim3(256), 0, st, a); };
    if (a.near_stride) return a.rank == 3 ? run(k_near<3, true>) : run(k_near<2, true>);
    return a.rank == 3 ? run(k_near<3, false>) : run(k_near<2, false>);
}

cudaError_t launch_local_expand(const LocalArgs& a, int mode, cudaStream_t st)
{
    auto run = [&](auto kern) {
        return launch_chained(kern, dim3(one_wave(kern)), dim3(256), 0, st, a, mode);
    };
    if (a.rank == 3) return a.vec ? run(k_expand<3, true>) : run(k_expand<3, false>);
    return a.vec ? run(k_expand<2, true>) : run(k_expand<2, false>);
}

cudaError_t launch_host_fixup(const LocalArgs& a, float* h_out_mapped, cudaStream_t st)
{
    const int vec = (a.nx % 4 == 0) && (reinterpret_cast<uintptr_t>(h_out_mapped) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(a.out) & 15) == 0;
    return launch_chained(k_host_fixup, dim3(one_wave(k_host_fixup)), dim3(256), 0, st, a, h_out_mapped, vec);
}

cudaError_t launch_local_pack_s(const LocalArgs& a, bool gated, cudaStream_t st)
{
    return launch_chained(k_pack_s, dim3(one_wave(k_pack_s)), dim3(256), 0, st, a, gated ? 1 : 0);
}

namespace {
// Grouped kernels over fields of either rank (and either load width): the
// body instance is picked per work item from the field's arguments.
__global__ void __launch_bounds__(256, QAI_DETECT_MINB) k_detect_group(const __grid_constant__ GroupQueue q, int mode)
{
    run_group<LocalArgs>(q, [&](const LocalArgs& a, int b, int n) {
        if (a.rank == 3) {
            if (a.vec) k_detect_body<3, true>(a, mode, b, n);
            else k_detect_body<3, false>(a, mode, b, n);
        } else {
            if (a.vec) k_detect_body<2, true>(a, mode, b, n);
            else k_detect_body<2, false>(a, mode, b, n);
        }
    });
}

__global__ void __launch_bounds__(256, QAI_NEAR_MINB) k_near_group(const __grid_constant__ GroupQueue q)
{
    run_group<LocalArgs>(q, [&](const LocalArgs& a, int b, int n) {
        if (a.rank == 3) k_near_body<3>(a, b, n);
        else k_near_body<2>(a, b, n);
    });
}

__global__ void __launch_bounds__(256) k_expand_group(const __grid_constant__ GroupQueue q, int mode)
{
    run_group<LocalArgs>(q, [&](const LocalArgs& a, int b, int n) {
        if (a.rank == 3) {
            if (a.vec) k_expand_body<3, true>(a, mode, b, n);
            else k_expand_body<3, false>(a, mode, b, n);
        } else {
            if (a.vec) k_expand_body<2, true>(a, mode, b, n);
            else k_expand_body<2, false>(a, mode, b, n);
        }
    });
}

__global__ void __launch_bounds__(256) k_pack_s_group(const __grid_constant__ GroupQueue q, int gated)
{
    run_group<LocalArgs>(q, [&](const LocalArgs& a, int b, int n) { k_pack_s_body(a, gated, b, n); });
}

template <class K, class... A>
cudaError_t run_grouped(K kern, const GroupQueue& q, cudaStream_t st, A... extra)
{
    const int grid = std::min(group_total(q), persistent_grid(kern, 256, 0));
    if (grid < 1) return cudaSuccess;
    return launch_chained(kern, dim3(grid), dim3(256), 0, st, q, extra...);
}
}  // namespace

cudaError_t launch_group_detect(const GroupQueue& q, int mode, cudaStream_t st)
{
    return run_grouped(k_detect_group, q, st, mode);
}

cudaError_t launch_group_near(const GroupQueue& q, cudaStream_t st) { return run_grouped(k_near_group, q, st); }

cudaError_t launch_group_expand(const GroupQueue& q, int mode, cudaStream_t st)
{
    return run_grouped(k_expand_group, q, st, mode);
}

cudaError_t launch_group_pack_s(const GroupQueue& q, int gated, cudaStream_t st)
{
    return run_grouped(k_pack_s_group, q, st, gated);
}

}  // namespace qai
