// qai_rowpass.cu -- row kernels: boundary detection fused with the first
// (x-axis) pass of each exact EDT.
//
// Phase 1 = step A (Algorithm 2, GetBoundaryAndSignMap) on the int32 index
// field q, then the x pass of the EDT of B1 (Algorithm 1 along x; with a
// binary input every parabola has g = 0, so the lower envelope reduces to the
// nearest site on the left and on the right, found by warp prefix scans).
// Phase 2 = GetBoundary(S) of Algorithm 3 (the sign-flipping boundary B2),
// then the x pass of the EDT of B2.
// For a rank-1 field the x pass is the last pass: phase 1 then writes Dist1
// and the propagated sign S (Algorithm 3), phase 2 writes D'' (step E).
//
// One warp owns one x-row. Three sweeps over the row, 32 points per step:
//   1. detect sites, keep a site byte per point in shared memory;
//   2. left to right: inclusive prefix max of site positions -> left site;
//   3. right to left: suffix min -> right site; the nearer one wins, the left
//      one on a tie (the smaller index, as Algorithm 1's strict query gives).
#include "qai_device.cuh"
#include "qai_launch.h"

namespace qai {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

template <int PHASE, bool FINAL>
__global__ void __launch_bounds__(256) k_rowpass(RowArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nx = a.nx;
    const int nxp = (nx + 31) & ~31;
    uint16_t* left = reinterpret_cast<uint16_t*>(smem) + warp * nxp;
    uint8_t* site = reinterpret_cast<uint8_t*>(reinterpret_cast<uint16_t*>(smem) + nwarps * nxp) +
                    warp * nxp;

    const int row = blockIdx.x * nwarps + warp;
    if (row >= a.nz * a.ny) return;  // whole warp leaves; only warp-level sync below
    const int z = row / a.ny;
    const int y = row - z * a.ny;
    const int base = row * nx;
    const int plane = a.ny * nx;
    bool row_inner = true;
    if (a.rank >= 2) row_inner = (y >= 1 && y <= a.ny - 2);
    if (a.rank >= 3) row_inner = row_inner && (z >= 1 && z <= a.nz - 2);

    // ---- sweep 1: site detection ------------------------------------------
    for (int x0 = 0; x0 < nx; x0 += 32) {
        const int x = x0 + lane;
        if (x >= nx) continue;
        const int i = base + x;
        const bool inner = row_inner && x >= 1 && x <= nx - 2;
        uint8_t f = 0;
        if (PHASE == 1) {
            uint8_t mask = 0;
            if (inner) {
                const int32_t q0 = a.q[i];
                int64_t sum = 0;
                int first = 0;
                bool differs = false, fast = false;
                // neighbours in the order z-, z+, y-, y+, x-, x+ (mask bits 0..5)
                auto visit = [&](int32_t lo, int32_t hi, int bit) {
                    const int64_t dl = (int64_t)lo - q0, dh = (int64_t)hi - q0;
                    if (dl == 0) mask |= (uint8_t)(1u << bit);
                    else { differs = true; if (!first) first = dl > 0 ? 1 : -1; }
                    if (dh == 0) mask |= (uint8_t)(1u << (bit + 1));
                    else { differs = true; if (!first) first = dh > 0 ? 1 : -1; }
                    sum += dl + dh;
                    int64_t g = (int64_t)hi - lo;
                    g = g < 0 ? -g : g;
                    if (g >= a.m.grad_threshold) fast = true;
                };
                if (a.rank >= 3) visit(a.q[i - plane], a.q[i + plane], 0);
                if (a.rank >= 2) visit(a.q[i - nx], a.q[i + nx], 2);
                visit(a.q[i - 1], a.q[i + 1], 4);
                if (differs) {
                    int sg = a.m.sign_rule == 1 ? first : (sum > 0) - (sum < 0);
                    if (fast) sg = 0;
                    f = (uint8_t)(1u | (sign_code(sg) << 1));
                }
            }
            a.eqm[i] = mask;
            if (a.dbg_b1) a.dbg_b1[i] = f & 1u;
            if (a.dbg_sb) a.dbg_sb[i] = (int8_t)sign_of_code(f >> 1);
        } else {
            if (inner) {
                const int s0 = a.s_in[i];
                const unsigned mask = a.eqm[i];
                const bool literal = a.m.b2_rule == 1;
                bool b2 = false;
                auto check = [&](int sn, int bit) {
                    if ((literal || ((mask >> bit) & 1u)) && sn != s0) b2 = true;
                };
                if (a.rank >= 3) { check(a.s_in[i - plane], 0); check(a.s_in[i + plane], 1); }
                if (a.rank >= 2) { check(a.s_in[i - nx], 2); check(a.s_in[i + nx], 3); }
                check(a.s_in[i - 1], 4);
                check(a.s_in[i + 1], 5);
                f = b2 ? 1 : 0;
            }
            if (a.dbg_b2) a.dbg_b2[i] = f;
        }
        site[x] = f;
    }
    __syncwarp();

    // ---- sweep 2: nearest site at or left of x -----------------------------
    int carry = -1;
    for (int x0 = 0; x0 < nx; x0 += 32) {
        const int x = x0 + lane;
        int v = (x < nx && (site[x] & 1u)) ? x : -1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v = max(v, t);
        }
        v = max(v, carry);
        if (x < nx) left[x] = v < 0 ? kInf16 : (uint16_t)v;
        carry = __shfl_sync(kFull, v, 31);
    }
    __syncwarp();

    // ---- sweep 3: nearest site at or right of x; emit ----------------------
    constexpr int kBig = 0x7FFFFFFF;
    carry = kBig;
    for (int x0 = (nx - 1) & ~31; x0 >= 0; x0 -= 32) {
        const int x = x0 + lane;
        int v = (x < nx && (site[x] & 1u)) ? x : kBig;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_down_sync(kFull, v, o);
            if (lane + o < 32) v = min(v, t);
        }
        v = min(v, carry);
        carry = __shfl_sync(kFull, v, 0);
        if (x >= nx) continue;
        const int i = base + x;
        const int lft = left[x];
        const int dl = lft != kInf16 ? x - lft : kBig;
        const int dr = v != kBig ? v - x : kBig;
        const bool valid = dl != kBig || dr != kBig;
        const int s = dl <= dr ? lft : v;   // tie -> left (smaller index)
        const int d = dl <= dr ? dl : dr;
        if (PHASE == 1) {
            const int code = valid ? (site[s] >> 1) & 3 : 0;
            if (!FINAL) {
                a.xw[i] = valid ? (uint16_t)((d << 2) | code) : kInf16;
            } else {
                a.dist1[i] = valid ? d * d : kDistInf;
                a.s_out[i] = (int8_t)sign_of_code(code);
            }
            if (a.dbg_idx) a.dbg_idx[i] = valid ? base + s : -1;
        } else {
            if (!FINAL) {
                a.xw[i] = valid ? (uint16_t)d : kInf16;
            } else {
                const int32_t d2 = valid ? d * d : kDistInf;
                a.out[i] = compensate(a.q[i], a.dist1_in[i], d2, a.s_in[i], a.m);
                if (a.dbg_dist2) a.dbg_dist2[i] = d2;
            }
        }
    }
}

}  // namespace

int rowpass_warps(int nx)
{
    const int nxp = (nx + 31) & ~31;
    int w = (200 * 1024) / (3 * nxp);
    return w < 1 ? 1 : (w > 8 ? 8 : w);
}

size_t rowpass_smem(int nx, int warps)
{
    const size_t nxp = (size_t)((nx + 31) & ~31);
    return (size_t)warps * nxp * 3;
}

cudaError_t launch_rowpass(int phase, bool final_pass, const RowArgs& a, cudaStream_t st)
{
    const int warps = rowpass_warps(a.nx);
    const size_t smem = rowpass_smem(a.nx, warps);
    const int rows = a.nz * a.ny;
    const dim3 grid((rows + warps - 1) / warps), block(32 * warps);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, block, smem, st>>>(a);
        return cudaGetLastError();
    };
    if (phase == 1) return final_pass ? go(k_rowpass<1, true>) : go(k_rowpass<1, false>);
    return final_pass ? go(k_rowpass<2, true>) : go(k_rowpass<2, false>);
}

}  // namespace qai
