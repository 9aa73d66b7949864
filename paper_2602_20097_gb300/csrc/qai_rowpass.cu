// qai_rowpass.cu -- row kernels: boundary detection fused with the first
// (x-axis) pass of each exact EDT.
//
// Phase 1 = step A (Algorithm 2, GetBoundaryAndSignMap) on the int32 index
// field q, then the x pass of the EDT of B1 (Algorithm 1 along x; with a
// binary input every parabola has g = 0, so the lower envelope reduces to the
// nearest site on the left and on the right).
// Phase 2 = GetBoundary(S) of Algorithm 3 (the sign-flipping boundary B2),
// then the x pass of the EDT of B2.
// For a rank-1 field the x pass is the last pass: phase 1 then writes Dist1
// and the propagated sign S (Algorithm 3), phase 2 writes D'' (step E).
//
// One warp owns one x-row and walks it in segments of 128 points, each lane
// holding 4 consecutive points (128-bit loads of q, 32-bit loads of the sign
// bytes). Two sweeps:
//   A  detect the sites of the segment; keep, per lane, a 4-bit site nibble
//      and the four 2-bit sign codes in shared memory, and the first and last
//      site of the segment;
//   B  nearest site to the left and to the right of every point: inside the
//      lane by a chain over its nibble, across lanes by a ballot and one
//      shuffle, across segments by carries (the right carry comes from a
//      backward scan over the segment summaries). The nearer site wins, the
//      left one on a tie (the smaller index, as Algorithm 1's strict query).
// Arithmetic on q is 32-bit; a warp whose loaded values reach |q| >= 2^27
// (where a sum of six differences could overflow) takes a 64-bit path.
#include <algorithm>

#include "qai_detect.cuh"
#include "qai_device.cuh"
#include "qai_launch.h"

namespace qai {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kSeg = 128;                 // points per warp step
constexpr int kNoneL = -(1 << 20);        // "no site on the left" position
constexpr int kNoneR = (1 << 20);         // "no site on the right" position
constexpr int kNoRef = (int)0x80000000;   // segment without a site

// Shared memory of one warp: three int arrays of segment summaries and the
// per-lane site nibbles / sign codes (one u16 per 4 points).
__host__ __device__ inline size_t smem_per_warp(int nx)
{
    const size_t nseg = (size_t)((nx + kSeg - 1) / kSeg);
    return ((nseg * 3 * 4 + nseg * 32 * 2) + 15) & ~(size_t)15;
}

// Shared memory of a CTA that walks one row with all its warps: the warp
// layout plus, per segment, the last site left of it.
__host__ __device__ inline size_t smem_coop(int nx)
{
    const size_t nseg = (size_t)((nx + kSeg - 1) / kSeg);
    return ((nseg * 4 * 4 + nseg * 32 * 2) + 15 + 16) & ~(size_t)15;
}

// A site reference packs the position and the 2-bit sign code.
__device__ __forceinline__ int make_ref(int pos, int code) { return (pos << 2) | code; }

struct RowSmem {
    uint16_t* info;   // [nseg * 32]: bits 0..3 site nibble, 4..11 sign codes
    int* sfirst;      // [nseg] first site ref of the segment (kNoRef if none)
    int* slast;       // [nseg] last site ref
    int* nextr;       // [nseg] first site ref right of the segment
};

__device__ __forceinline__ uint32_t load4_u8(const void* base, int x0, int nx, bool vec)
{
    const uint8_t* p = static_cast<const uint8_t*>(base);
    if (vec) return x0 < nx ? __ldg(reinterpret_cast<const uint32_t*>(p + x0)) : 0u;
    uint32_t w = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (x0 + j < nx) w |= (uint32_t)__ldg(p + x0 + j) << (8 * j);
    return w;
}

// One warp's work: x-row `row` of the field `a`, with `wsm` this warp's
// shared memory (smem_per_warp of an extent >= a.nx). COOP: every warp of
// the CTA walks the same row (segments dealt round robin; `wsm` is the CTA's
// smem_coop of an extent >= a.nx): the segments are independent but for the
// value left of each (loaded directly) and the sites outside them (the
// segment summaries, combined by one thread between the sweeps). Every
// thread of the CTA must call it.
template <int PHASE, int RANK, bool FINAL, bool DEBUG, bool VEC, bool COOP = false>
__device__ __forceinline__ void rowpass_row(const RowArgs& a, const int row, unsigned char* wsm)
{
    const int lane = threadIdx.x & 31;
    const int nx = a.nx;
    const int nseg = (nx + kSeg - 1) / kSeg;
    const int seg0 = COOP ? (int)(threadIdx.x >> 5) : 0;
    const int segstep = COOP ? (int)(blockDim.x >> 5) : 1;
    RowSmem sm;
    sm.sfirst = reinterpret_cast<int*>(wsm);
    sm.slast = sm.sfirst + nseg;
    sm.nextr = sm.slast + nseg;
    int* carryl = sm.nextr + nseg;  // COOP: the last site left of each segment
    sm.info = reinterpret_cast<uint16_t*>(COOP ? carryl + nseg : sm.nextr + nseg);
    int* s_rowfirst = reinterpret_cast<int*>(sm.info + nseg * 32);  // COOP: the first site of the row
    const int z = row / a.ny;
    const int y = row - z * a.ny;
    const int rbase = row * nx;
    const int plane = a.ny * nx;
    bool row_inner = true;
    if (RANK >= 2) row_inner = (y >= 1 && y <= a.ny - 2);
    if (RANK >= 3) row_inner = row_inner && (z >= 1 && z <= a.nz - 2);

    // ---- sweep A: sites of each segment ------------------------------------
    int carry_prev = 0;  // value left of the segment (phase 1: q, phase 2: S byte)
    for (int seg = seg0; seg < nseg; seg += segstep) {
        const int x0 = seg * kSeg + 4 * lane;
        unsigned nib = 0, codes = 0;
        if (COOP && lane == 0 && x0 > 0) {  // the value left of the segment, from memory
            if (PHASE == 1) carry_prev = __ldg(a.q + rbase + x0 - 1);
            else carry_prev = (int)((uint32_t)__ldg(reinterpret_cast<const uint8_t*>(a.s_in) + rbase + x0 - 1) << 24);
        }
        if (PHASE == 1) {
            int c[4], yl[4] = {0, 0, 0, 0}, yr[4] = {0, 0, 0, 0}, zl[4] = {0, 0, 0, 0},
                      zr[4] = {0, 0, 0, 0};
            load4_i32(a.q + rbase, x0, nx, VEC, c);
            int xm = __shfl_up_sync(kFull, c[3], 1);
            int xp = __shfl_down_sync(kFull, c[0], 1);
            const int last_c3 = __shfl_sync(kFull, c[3], 31);
            if (lane == 0) xm = carry_prev;
            if (lane == 31) xp = (x0 + 4 < nx) ? __ldg(a.q + rbase + x0 + 4) : 0;
            carry_prev = last_c3;
            unsigned eq = 0;
            if (row_inner) {
                if (RANK >= 2) {
                    load4_i32(a.q + rbase - nx, x0, nx, VEC, yl);
                    load4_i32(a.q + rbase + nx, x0, nx, VEC, yr);
                }
                if (RANK >= 3) {
                    load4_i32(a.q + rbase - plane, x0, nx, VEC, zl);
                    load4_i32(a.q + rbase + plane, x0, nx, VEC, zr);
                }
                // 32-bit arithmetic is exact while every |q| < 2^27
                unsigned acc = (unsigned)(xm ^ (xm >> 31)) | (unsigned)(xp ^ (xp >> 31));
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc |= (unsigned)(c[j] ^ (c[j] >> 31)) | (unsigned)(yl[j] ^ (yl[j] >> 31)) |
                           (unsigned)(yr[j] ^ (yr[j] >> 31)) | (unsigned)(zl[j] ^ (zl[j] >> 31)) |
                           (unsigned)(zr[j] ^ (zr[j] >> 31));
                }
                const bool wide = __any_sync(kFull, acc >= (1u << 27));
                if (!wide && a.m.sign_rule == 0) {
                    const int thm1 = a.m.grad_threshold - 1;
                    const unsigned lim = 2u * (unsigned)thm1;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int x = x0 + j;
                        const bool inner = x >= 1 && x <= nx - 2;
                        unsigned mk, st, cd;
                        detect_sum32<RANK>(c[j], zl[j], zr[j], yl[j], yr[j], j == 0 ? xm : c[j - 1],
                                           j == 3 ? xp : c[j + 1], inner, thm1, lim, mk, st, cd);
                        eq |= mk << (8 * j);
                        nib |= st << j;
                        codes |= cd << (2 * j);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int x = x0 + j;
                        const bool inner = x >= 1 && x <= nx - 2;
                        const int l = j == 0 ? xm : c[j - 1];
                        const int r = j == 3 ? xp : c[j + 1];
                        unsigned mk;
                        bool site;
                        int code;
                        if (!wide)
                            detect_point<RANK, false>(c[j], zl[j], zr[j], yl[j], yr[j], l, r, inner, a.m, mk, site, code);
                        else
                            detect_point<RANK, true>(c[j], zl[j], zr[j], yl[j], yr[j], l, r, inner, a.m, mk, site, code);
                        eq |= mk << (8 * j);
                        nib |= (unsigned)site << j;
                        codes |= (unsigned)code << (2 * j);
                    }
                }
                // off the interior along x nothing is on B1: the all-equal
                // mask there (readers take B1 from a clear bit)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (x0 + j == 0 || x0 + j == nx - 1) eq = (eq & ~(0xFFu << (8 * j))) | (0x3Fu << (8 * j));
                if (VEC) {
                    if (x0 < nx) *reinterpret_cast<uint32_t*>(a.eqm + rbase + x0) = eq;
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (x0 + j < nx) a.eqm[rbase + x0 + j] = (uint8_t)(eq >> (8 * j));
                }
            } else {
                // rows off the interior: nothing is on B1, the all-equal mask
                if (VEC) {
                    if (x0 < nx) *reinterpret_cast<uint32_t*>(a.eqm + rbase + x0) = 0x3F3F3F3Fu;
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (x0 + j < nx) a.eqm[rbase + x0 + j] = 0x3Fu;
                }
            }
            if (a.out_pre) {
                // the output wherever Dist2 does not matter: on B1 the weight
                // is 1 (C = S_B eta eps), elsewhere D' until a later kernel
                // writes the points with S != 0; the same expressions as
                // compensate(), so the same bits
                float o[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned cd = (codes >> (2 * j)) & 3u;
                    const float cc = (cd == 1u ? 1.0f : (cd == 2u ? -1.0f : 0.0f)) * a.m.eta_eb;
                    o[j] = a.m.output_c ? cc : fmaf((float)c[j], a.m.two_eb, cc);
                }
                if (VEC) {
                    if (x0 < nx) *reinterpret_cast<float4*>(a.out_pre + rbase + x0) = make_float4(o[0], o[1], o[2], o[3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (x0 + j < nx) a.out_pre[rbase + x0 + j] = o[j];
                }
            }
            if (DEBUG) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (x0 + j >= nx) continue;
                    if (a.dbg_b1) a.dbg_b1[rbase + x0 + j] = (nib >> j) & 1u;
                    if (a.dbg_sb) a.dbg_sb[rbase + x0 + j] = (int8_t)sign_of_code((codes >> (2 * j)) & 3u);
                }
            }
        } else {
            // GetBoundary(S): B2 where an axis neighbour (with the same q under
            // SAME_Q) has a different S; four points per 32-bit word.
            const uint32_t cw = load4_u8(a.s_in + rbase, x0, nx, VEC);
            uint32_t xmw = __shfl_up_sync(kFull, cw, 1);
            uint32_t xpw = __shfl_down_sync(kFull, cw, 1);
            const uint32_t last_w = __shfl_sync(kFull, cw, 31);
            if (lane == 0) xmw = (uint32_t)carry_prev;
            if (lane == 31) xpw = (x0 + 4 < nx) ? (uint32_t)__ldg(reinterpret_cast<const uint8_t*>(a.s_in) + rbase + x0 + 4) : 0u;
            carry_prev = (int)last_w;
            if (row_inner) {
                const uint32_t eqw = load4_u8(a.eqm + rbase, x0, nx, VEC);
                const bool literal = a.m.b2_rule == 1;
                // byte k of sel(bit) = 0xFF if bit `bit` of eqm byte k is set
                auto sel = [&](int bit) -> uint32_t {
                    return literal ? 0xFFFFFFFFu : __vcmpne4(eqw & (0x01010101u << bit), 0u);
                };
                uint32_t b2 = (__vcmpne4(__byte_perm(xmw, cw, 0x6543), cw) & sel(4)) |
                              (__vcmpne4(__byte_perm(cw, xpw, 0x4321), cw) & sel(5));
                if (RANK >= 2) {
                    b2 |= (__vcmpne4(load4_u8(a.s_in + rbase - nx, x0, nx, VEC), cw) & sel(2)) |
                          (__vcmpne4(load4_u8(a.s_in + rbase + nx, x0, nx, VEC), cw) & sel(3));
                }
                if (RANK >= 3) {
                    b2 |= (__vcmpne4(load4_u8(a.s_in + rbase - plane, x0, nx, VEC), cw) & sel(0)) |
                          (__vcmpne4(load4_u8(a.s_in + rbase + plane, x0, nx, VEC), cw) & sel(1));
                }
                // gather the top bit of each byte into a nibble
                nib = ((b2 & 0x80808080u) * 0x00204081u) >> 28;
                // interior along x
                if (x0 == 0) nib &= ~1u;
                if (x0 + 4 > nx - 1) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (x0 + j > nx - 2) nib &= ~(1u << j);
                }
            }
            if (DEBUG && a.dbg_b2) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (x0 + j < nx) a.dbg_b2[rbase + x0 + j] = (nib >> j) & 1u;
            }
        }
        sm.info[seg * 32 + lane] = (uint16_t)(nib | (codes << 4));
        const unsigned H = __ballot_sync(kFull, nib != 0);
        const int my_first = nib ? make_ref(x0 + __ffs(nib) - 1, (codes >> (2 * (__ffs(nib) - 1))) & 3u) : 0;
        const int my_last = nib ? make_ref(x0 + 31 - __clz(nib), (codes >> (2 * (31 - __clz(nib)))) & 3u) : 0;
        const int f = __shfl_sync(kFull, my_first, H ? __ffs(H) - 1 : 0);
        const int l = __shfl_sync(kFull, my_last, H ? 31 - __clz(H) : 0);
        if (lane == 0) {
            sm.sfirst[seg] = H ? f : kNoRef;
            sm.slast[seg] = H ? l : kNoRef;
        }
    }
    int row_first = kNoRef;  // first site of the row
    if (COOP) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int nxt = kNoRef, prv = kNoRef;
            for (int seg = nseg - 1; seg >= 0; --seg) {
                sm.nextr[seg] = nxt;
                if (sm.sfirst[seg] != kNoRef) nxt = sm.sfirst[seg];
            }
            for (int seg = 0; seg < nseg; ++seg) {
                carryl[seg] = prv;
                if (sm.slast[seg] != kNoRef) prv = sm.slast[seg];
            }
            *s_rowfirst = nxt;
        }
        __syncthreads();
        row_first = *s_rowfirst;
    } else {
        __syncwarp();
        if (lane == 0) {
            int nxt = kNoRef;
            for (int seg = nseg - 1; seg >= 0; --seg) {
                sm.nextr[seg] = nxt;
                if (sm.sfirst[seg] != kNoRef) nxt = sm.sfirst[seg];
            }
            row_first = nxt;
        }
        __syncwarp();
        row_first = __shfl_sync(kFull, row_first, 0);
    }
    // a row without sites (common for the sparse sign flips of the second
    // EDT) is INF everywhere: no sweep B
    if (!FINAL && !DEBUG && row_first == kNoRef) {
        for (int seg = seg0; seg < nseg; seg += segstep) {
            const int x0 = seg * kSeg + 4 * lane;
            if (VEC) {
                if (x0 < nx) *reinterpret_cast<uint2*>(a.xw + rbase + x0) = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (x0 + j < nx) a.xw[rbase + x0 + j] = (uint16_t)kInf16;
            }
        }
        return;
    }

    // ---- sweep B: nearest site on both sides; emit -------------------------
    const unsigned lt = (1u << lane) - 1u;
    const unsigned gt = ~((2u << lane) - 1u);
    int carry_l = kNoRef;
    for (int seg = seg0; seg < nseg; seg += segstep) {
        const int x0 = seg * kSeg + 4 * lane;
        if (COOP) carry_l = carryl[seg];
        const unsigned v = sm.info[seg * 32 + lane];
        const unsigned nib = v & 15u, codes = v >> 4;
        const unsigned H = __ballot_sync(kFull, nib != 0);
        const int my_first = nib ? make_ref(x0 + __ffs(nib) - 1, (codes >> (2 * (__ffs(nib) - 1))) & 3u) : 0;
        const int my_last = nib ? make_ref(x0 + 31 - __clz(nib), (codes >> (2 * (31 - __clz(nib)))) & 3u) : 0;
        const unsigned below = H & lt, above = H & gt;
        const int lsrc = below ? 31 - __clz(below) : lane;
        const int rsrc = above ? __ffs(above) - 1 : lane;
        const int lv = __shfl_sync(kFull, my_last, lsrc);
        const int rv = __shfl_sync(kFull, my_first, rsrc);
        int lref = below ? lv : carry_l;
        int rref = above ? rv : sm.nextr[seg];
        if (H) carry_l = sm.slast[seg];
        // chains over the lane's own four points
        int L[4], R[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if ((nib >> j) & 1u) lref = make_ref(x0 + j, (codes >> (2 * j)) & 3u);
            L[j] = lref;
        }
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            if ((nib >> j) & 1u) rref = make_ref(x0 + j, (codes >> (2 * j)) & 3u);
            R[j] = rref;
        }
        uint32_t packed[2] = {0u, 0u};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = x0 + j;
            const int lp = L[j] == kNoRef ? kNoneL : (L[j] >> 2);
            const int rp = R[j] == kNoRef ? kNoneR : (R[j] >> 2);
            const int dl = x - lp, dr = rp - x;
            const bool left = dl <= dr;
            const int d = left ? dl : dr;
            const int ref = left ? L[j] : R[j];
            const bool valid = d < (1 << 19);
            const int code = ref & 3;
            if (PHASE == 1) {
                if (!FINAL) {
                    const uint32_t w = valid ? (uint32_t)((d << 2) | code) : kInf16;
                    packed[j >> 1] |= w << (16 * (j & 1));
                } else if (x < nx) {
                    a.dist1[rbase + x] = valid ? d * d : kDistInf;
                    a.s_out[rbase + x] = (int8_t)sign_of_code(valid ? code : 0);
                }
                if (DEBUG && a.dbg_idx && x < nx) a.dbg_idx[rbase + x] = valid ? rbase + (ref >> 2) : -1;
            } else {
                if (!FINAL) {
                    const uint32_t w = valid ? (uint32_t)d : kInf16;
                    packed[j >> 1] |= w << (16 * (j & 1));
                } else if (x < nx) {
                    const int32_t d2 = valid ? d * d : kDistInf;
                    a.out[rbase + x] = compensate(a.q[rbase + x], a.dist1_in[rbase + x], d2,
                                                  a.s_in[rbase + x], a.m);
                    if (DEBUG && a.dbg_dist2) a.dbg_dist2[rbase + x] = d2;
                }
            }
        }
        if (!FINAL) {
            if (VEC) {
                if (x0 < nx) *reinterpret_cast<uint2*>(a.xw + rbase + x0) = make_uint2(packed[0], packed[1]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (x0 + j < nx) a.xw[rbase + x0 + j] = (uint16_t)(packed[j >> 1] >> (16 * (j & 1)));
            }
        }
    }
}

template <int PHASE, int RANK, bool FINAL, bool DEBUG, bool VEC>
__device__ __forceinline__ void k_rowpass_body(const RowArgs& a, const int bx, const int gx)
{
    extern __shared__ __align__(16) unsigned char smem[];
    wait_prior_grid();
    // gated launches (signed-point route): run only when the flag is set
    if (a.gate && *static_cast<const volatile int*>(a.gate) == 0) return;
    // row pass 1 of the route starts its counters again (not the timeout and
    // local-EDT flags)
    if (PHASE == 1 && a.route_ctr && bx == 0 && threadIdx.x < kCtrTimeout)
        a.route_ctr[threadIdx.x] = 0;
    const int warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    // one row per warp, or (a grid smaller than the rows: the dense second EDT
    // behind the signed-point route) a loop over them; only warp-level sync
    for (int row = bx * warps + warp; row < a.nz * a.ny; row += gx * warps) {
        rowpass_row<PHASE, RANK, FINAL, DEBUG, VEC>(a, row, smem + (size_t)warp * smem_per_warp(a.nx));
        __syncwarp();
    }
}

template <int PHASE, int RANK, bool FINAL, bool DEBUG, bool VEC>
__global__ void __launch_bounds__(256) k_rowpass(RowArgs a)
{
    k_rowpass_body<PHASE, RANK, FINAL, DEBUG, VEC>(a, blockIdx.x, gridDim.x);
}

// Long rows and few of them (2-D fields, 1-D fields): a CTA per row, all its
// warps on that row.
template <int PHASE, int RANK, bool FINAL, bool DEBUG, bool VEC>
__global__ void __launch_bounds__(512) k_rowpass_coop(RowArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    wait_prior_grid();
    if (a.gate && *static_cast<const volatile int*>(a.gate) == 0) return;
    if (PHASE == 1 && a.route_ctr && blockIdx.x == 0 && threadIdx.x < kCtrTimeout)
        a.route_ctr[threadIdx.x] = 0;
    for (int row = blockIdx.x; row < a.nz * a.ny; row += gridDim.x) {
        rowpass_row<PHASE, RANK, FINAL, DEBUG, VEC, true>(a, row, smem);
        __syncthreads();
    }
}


// Several fields in one launch: global row g belongs to field f with
// first_row[f] <= g < first_row[f + 1]; the table travels by value.
template <int PHASE, int RANK, bool FINAL>
__global__ void __launch_bounds__(256) k_rowpass_grouped(const __grid_constant__ RowTable t)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int g = blockIdx.x * t.warps + warp;
    if (g >= t.first_row[t.n]) return;
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.first_row[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    const RowArgs& a = t.args[lo];
    unsigned char* wsm = smem + (size_t)warp * smem_per_warp(t.smem_nx);
    if (a.vec) rowpass_row<PHASE, RANK, FINAL, false, true>(a, g - t.first_row[lo], wsm);
    else rowpass_row<PHASE, RANK, FINAL, false, false>(a, g - t.first_row[lo], wsm);
}

// A CTA of 16 warps per row when the rows are long and too few for one warp
// each to fill the GPU.
constexpr int kCoopWarps = 16;
bool use_coop(const RowArgs& a, int sms)
{
    const int nseg = (a.nx + kSeg - 1) / kSeg;
    return nseg >= 8 && (int64_t)a.nz * a.ny < (int64_t)sms * 32;
}

template <int PHASE, int RANK, bool FINAL>
cudaError_t go_coop(const RowArgs& a, bool debug, bool vec, int sms, cudaStream_t st)
{
    const size_t smem = smem_coop(a.nx);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * kCoopWarps, smem) != cudaSuccess || per < 1)
            per = 1;
        const int rows = a.nz * a.ny;
        const int grid = std::max(1, std::min(rows, sms * per));
        return launch_chained(kern, dim3(grid), dim3(32 * kCoopWarps), smem, st, a);
    };
    if (debug) return vec ? run(k_rowpass_coop<PHASE, RANK, FINAL, true, true>)
                          : run(k_rowpass_coop<PHASE, RANK, FINAL, true, false>);
    return vec ? run(k_rowpass_coop<PHASE, RANK, FINAL, false, true>)
               : run(k_rowpass_coop<PHASE, RANK, FINAL, false, false>);
}

template <int PHASE, int RANK, bool FINAL>
cudaError_t go(const RowArgs& a, bool debug, bool vec, dim3 grid, dim3 block, size_t smem,
               cudaStream_t st)
{
    {
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (use_coop(a, sms)) return go_coop<PHASE, RANK, FINAL>(a, debug, vec, sms, st);
    }
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        dim3 g = grid;
        if (a.gate) {  // gated: a resident grid that loops over the rows
            int dev = 0, sms = 152, per = 1;
            if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, (int)block.x, smem) != cudaSuccess || per < 1)
                per = 1;
            g.x = std::min<unsigned>(g.x, (unsigned)(sms * per));
        }
        return launch_chained(kern, g, block, smem, st, a);
    };
    if (debug) return vec ? run(k_rowpass<PHASE, RANK, FINAL, true, true>)
                          : run(k_rowpass<PHASE, RANK, FINAL, true, false>);
    return vec ? run(k_rowpass<PHASE, RANK, FINAL, false, true>)
               : run(k_rowpass<PHASE, RANK, FINAL, false, false>);
}

}  // namespace

int rowpass_warps(int nx)
{
    const size_t per = smem_per_warp(nx);
    int w = (int)((96 * 1024) / per);
    return w < 1 ? 1 : (w > 8 ? 8 : w);
}

size_t rowpass_smem(int nx, int warps) { return (size_t)warps * smem_per_warp(nx); }

void prepare_rowpass(RowArgs& a)
{
    // 128-bit / 32-bit accesses need 4 | nx and 16-byte aligned base pointers
    auto al = [](const void* p, int b) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) % b) == 0; };
    a.vec = (a.nx % 4 == 0) && al(a.q, 16) && al(a.eqm, 4) && al(a.s_in, 4) && al(a.xw, 8) &&
            al(a.out_pre, 16);
}

cudaError_t launch_rowpass_grouped(int phase, bool final_pass, const RowTable& t, cudaStream_t st)
{
    const size_t smem = rowpass_smem(t.smem_nx, t.warps);
    const int rows = t.first_row[t.n];
    const dim3 grid((rows + t.warps - 1) / t.warps), block(32 * t.warps);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, block, smem, st>>>(t);
        return cudaGetLastError();
    };
    const int rank = t.args[0].rank;
    if (phase == 1) {
        if (final_pass) return run(k_rowpass_grouped<1, 1, true>);
        return rank == 2 ? run(k_rowpass_grouped<1, 2, false>) : run(k_rowpass_grouped<1, 3, false>);
    }
    if (final_pass) return run(k_rowpass_grouped<2, 1, true>);
    return rank == 2 ? run(k_rowpass_grouped<2, 2, false>) : run(k_rowpass_grouped<2, 3, false>);
}

namespace {
// Grouped row passes of rank-2 and rank-3 fields (non-final): the body
// instance is picked per work item from the field's arguments.
template <int PHASE>
__global__ void __launch_bounds__(256) k_rowpass_group(const __grid_constant__ GroupQueue q)
{
    run_group<RowArgs>(q, [&](const RowArgs& a, int b, int n) {
        if (a.rank == 3) {
            if (a.vec) k_rowpass_body<PHASE, 3, false, false, true>(a, b, n);
            else k_rowpass_body<PHASE, 3, false, false, false>(a, b, n);
        } else {
            if (a.vec) k_rowpass_body<PHASE, 2, false, false, true>(a, b, n);
            else k_rowpass_body<PHASE, 2, false, false, false>(a, b, n);
        }
    });
}
}  // namespace

cudaError_t launch_group_rowpass(const GroupQueue& q, int phase, int warps, int max_nx, cudaStream_t st)
{
    const size_t smem = rowpass_smem(max_nx, warps);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int grid = std::min(group_total(q), persistent_grid(kern, 32 * warps, smem));
        if (grid < 1) return cudaSuccess;
        return launch_chained(kern, dim3(grid), dim3(32 * warps), smem, st, q);
    };
    return phase == 1 ? run(k_rowpass_group<1>) : run(k_rowpass_group<2>);
}

cudaError_t launch_rowpass(int phase, bool final_pass, const RowArgs& a_in, bool debug, cudaStream_t st)
{
    RowArgs a = a_in;
    prepare_rowpass(a);
    const int warps = rowpass_warps(a.nx);
    const size_t smem = rowpass_smem(a.nx, warps);
    const int rows = a.nz * a.ny;
    const dim3 grid((rows + warps - 1) / warps), block(32 * warps);
    const bool vec = a.vec != 0;
    if (phase == 1) {
        if (final_pass) return go<1, 1, true>(a, debug, vec, grid, block, smem, st);
        if (a.rank == 2) return go<1, 2, false>(a, debug, vec, grid, block, smem, st);
        return go<1, 3, false>(a, debug, vec, grid, block, smem, st);
    }
    if (final_pass) return go<2, 1, true>(a, debug, vec, grid, block, smem, st);
    if (a.rank == 2) return go<2, 2, false>(a, debug, vec, grid, block, smem, st);
    return go<2, 3, false>(a, debug, vec, grid, block, smem, st);
}

}  // namespace qai
