// qai_detect.cuh -- step A (Algorithm 2, GetBoundaryAndSignMap) for one
// point, shared by the row pass and the local first EDT.
#pragma once
#include <cstdint>

#include "qai_device.cuh"

namespace qai {

// Four consecutive int32 values starting at p[x0] (zeros past nx); vec: one
// 128-bit load (x0 and p 16-byte aligned, nx a multiple of 4).
__device__ __forceinline__ void load4_i32(const int32_t* p, int x0, int nx, bool vec, int v[4])
{
    if (vec) {
        if (x0 < nx) {
            const int4 t = __ldg(reinterpret_cast<const int4*>(p + x0));
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
            v[0] = v[1] = v[2] = v[3] = 0;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = (x0 + j < nx) ? __ldg(p + x0 + j) : 0;
    }
}

// Step A for one point: the equal-q neighbour mask (bits z-, z+, y-, y+, x-,
// x+; absent axes count as equal), whether it is a boundary, its sign code.
template <int RANK, bool WIDE>
__device__ __forceinline__ void detect_point(int q0, int zl, int zr, int yl, int yr, int xl, int xr,
                                             bool inner, const MethodArgs& m, unsigned& mask,
                                             bool& site, int& code)
{
    mask = (unsigned)(xl == q0) << 4 | (unsigned)(xr == q0) << 5;
    if (RANK >= 2) mask |= (unsigned)(yl == q0) << 2 | (unsigned)(yr == q0) << 3;
    else mask |= 0xCu;
    if (RANK >= 3) mask |= (unsigned)(zl == q0) | (unsigned)(zr == q0) << 1;
    else mask |= 0x3u;
    site = inner && mask != 0x3Fu;
    int sg, first = 0;
    bool fast;
    if (!WIDE) {
        int sum = (xl - q0) + (xr - q0);
        const unsigned thm1 = (unsigned)m.grad_threshold - 1u, lim = 2u * thm1;
        fast = (unsigned)(xr - xl + (int)thm1) > lim;
        if (RANK >= 2) { sum += (yl - q0) + (yr - q0); fast |= (unsigned)(yr - yl + (int)thm1) > lim; }
        if (RANK >= 3) { sum += (zl - q0) + (zr - q0); fast |= (unsigned)(zr - zl + (int)thm1) > lim; }
        sg = (sum > 0) - (sum < 0);
        if (m.sign_rule == 1) {
            // first differing neighbour in the order z-, z+, y-, y+, x-, x+
            first = xr != q0 ? (xr > q0 ? 1 : -1) : 0;
            first = xl != q0 ? (xl > q0 ? 1 : -1) : first;
            if (RANK >= 2) {
                first = yr != q0 ? (yr > q0 ? 1 : -1) : first;
                first = yl != q0 ? (yl > q0 ? 1 : -1) : first;
            }
            if (RANK >= 3) {
                first = zr != q0 ? (zr > q0 ? 1 : -1) : first;
                first = zl != q0 ? (zl > q0 ? 1 : -1) : first;
            }
        }
    } else {
        const int64_t Q = q0;
        int64_t sum = ((int64_t)xl - Q) + ((int64_t)xr - Q);
        auto gr = [&](int lo, int hi) {
            int64_t g = (int64_t)hi - lo;
            return (g < 0 ? -g : g) >= (int64_t)m.grad_threshold;
        };
        fast = gr(xl, xr);
        if (RANK >= 2) { sum += ((int64_t)yl - Q) + ((int64_t)yr - Q); fast |= gr(yl, yr); }
        if (RANK >= 3) { sum += ((int64_t)zl - Q) + ((int64_t)zr - Q); fast |= gr(zl, zr); }
        sg = (sum > 0) - (sum < 0);
        if (m.sign_rule == 1) {
            first = xr != q0 ? (xr > q0 ? 1 : -1) : 0;
            first = xl != q0 ? (xl > q0 ? 1 : -1) : first;
            if (RANK >= 2) {
                first = yr != q0 ? (yr > q0 ? 1 : -1) : first;
                first = yl != q0 ? (yl > q0 ? 1 : -1) : first;
            }
            if (RANK >= 3) {
                first = zr != q0 ? (zr > q0 ? 1 : -1) : first;
                first = zl != q0 ? (zl > q0 ? 1 : -1) : first;
            }
        }
    }
    if (m.sign_rule == 1) sg = first;
    code = (site && !fast) ? sign_code(sg) : 0;
}

// The common case of detect_point: sign rule SUM and every |q| < 2^27, so
// that the sum of the neighbour differences fits 32 bits.
template <int RANK>
__device__ __forceinline__ void detect_sum32(int q0, int zl, int zr, int yl, int yr, int xl, int xr,
                                             bool inner, int thm1, unsigned lim, unsigned& mask,
                                             unsigned& site, unsigned& code)
{
    unsigned mk = (xl == q0 ? 0x10u : 0u) | (xr == q0 ? 0x20u : 0u);
    int sum = xl + xr;
    bool fast = (unsigned)(xr - xl + thm1) > lim;
    if (RANK >= 2) {
        mk |= (yl == q0 ? 0x4u : 0u) | (yr == q0 ? 0x8u : 0u);
        sum += yl + yr;
        fast |= (unsigned)(yr - yl + thm1) > lim;
    } else {
        mk |= 0xCu;
    }
    if (RANK >= 3) {
        mk |= (zl == q0 ? 0x1u : 0u) | (zr == q0 ? 0x2u : 0u);
        sum += zl + zr;
        fast |= (unsigned)(zr - zl + thm1) > lim;
    } else {
        mk |= 0x3u;
    }
    sum -= 2 * RANK * q0;
    const bool s = inner && mk != 0x3Fu;
    const unsigned cd = sum > 0 ? 1u : (sum < 0 ? 2u : 0u);
    code = (s && !fast) ? cd : 0u;
    site = s ? 1u : 0u;
    mask = mk;
}

}  // namespace qai
