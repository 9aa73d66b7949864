// qai_backward.cu -- adjoint of step E with the EDT assignment held fixed.
//
// D'' = D' + S w eta eps with w = 1 / (1 + (k1/k2)^p), k = sqrt(Dist). For a
// loss with dL/dD'' = G:
//   dL/dD'  = G
//   dL/deta = sum G S w eps
//   dL/dp   = sum G S eta eps w (1 - w) (ln k2 - ln k1)
// (w is constant where k1 = 0, k2 = 0 or k2 is infinite, so dw/dp = 0 there).
// One grid-stride pass: each thread sums its terms in fp32 with Kahan
// compensation and takes the sums to FP64 at the end; each block writes its
// two FP64 totals to a partials array, and a one-block kernel adds the
// partials in a fixed order, so the result is the same on every run.
#include <algorithm>

#include "qai_device.cuh"
#include "qai_launch.h"

namespace qai {
namespace {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

// The 2-bit fields of points i .. i + 3 (one row, 4 | nx) of a packed map
// with wpr words a row, in the low byte.
__device__ __forceinline__ unsigned packed4(const uint32_t* m, int wpr, int nx, int i)
{
    const int row = i / nx, x0 = i - row * nx;
    return (__ldg(m + (int64_t)row * wpr + (x0 >> 4)) >> (2 * (x0 & 15))) & 0xFFu;
}
// The 2-bit field of point i.
__device__ __forceinline__ unsigned packed1(const uint32_t* m, int wpr, int nx, int i)
{
    const int row = i / nx, x = i - row * nx;
    return (__ldg(m + (int64_t)row * wpr + (x >> 4)) >> (2 * (x & 15))) & 3u;
}
// S as -1, 0, +1 from its 2-bit code (0, 1: +1, 2: -1).
__device__ __forceinline__ int s_of(unsigned c) { return c == 1u ? 1 : (c == 2u ? -1 : 0); }

// vec: N a multiple of 4 and every array aligned for 4-point accesses (and,
// with the packed maps, 4 | nx).
__global__ void __launch_bounds__(256) k_backward(BackArgs a, int vec)
{
    GradAcc acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // Terms vanish where S = 0: Dist1, Dist2 (and G, unless dL/dD' is
    // wanted) are read only for groups of points with some S != 0.
    if (a.spk) {  // S and B1 from a plain forward's packed maps (dL/dD' copied by the host)
        if (vec) {
            for (int64_t i = t0; i < (a.N >> 2); i += stride) {
                const unsigned sc = packed4(a.spk, a.wpr, a.nx, (int)(4 * i));
                if (!sc) continue;
                const unsigned cc = packed4(a.codes, a.wpr, a.nx, (int)(4 * i));
                const float4 g = __ldg(reinterpret_cast<const float4*>(a.grad_out) + i);
                const int4 d1 = __ldg(reinterpret_cast<const int4*>(a.dist1) + i);
                const int4 d2 = __ldg(reinterpret_cast<const int4*>(a.dist2) + i);
                const float gv[4] = {g.x, g.y, g.z, g.w};
                const int d1v[4] = {d1.x, d1.y, d1.z, d1.w}, d2v[4] = {d2.x, d2.y, d2.z, d2.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int sv = s_of((sc >> (2 * j)) & 3u);
                    if (!sv) continue;
                    float te, tp;
                    grad_terms(gv[j], sv, ((cc >> (2 * j)) & 3u) ? 0 : d1v[j], d2v[j], a.p, te, tp);
                    acc.add(te, tp);
                }
            }
        } else {
            for (int64_t i = t0; i < a.N; i += stride) {
                const int sv = s_of(packed1(a.spk, a.wpr, a.nx, (int)i));
                if (!sv) continue;
                const int d1 = packed1(a.codes, a.wpr, a.nx, (int)i) ? 0 : __ldg(a.dist1 + i);
                float te, tp;
                grad_terms(__ldg(a.grad_out + i), sv, d1, __ldg(a.dist2 + i), a.p, te, tp);
                acc.add(te, tp);
            }
        }
    } else if (vec) {
        const int64_t n4 = a.N >> 2;
        for (int64_t i = t0; i < n4; i += stride) {
            const uint32_t sw = __ldg(reinterpret_cast<const uint32_t*>(a.s) + i);
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            if (sw || a.grad_dprime) g = __ldg(reinterpret_cast<const float4*>(a.grad_out) + i);
            if (a.grad_dprime) reinterpret_cast<float4*>(a.grad_dprime)[i] = g;
            if (!sw) continue;
            int4 d1 = __ldg(reinterpret_cast<const int4*>(a.dist1) + i);
            const int4 d2 = __ldg(reinterpret_cast<const int4*>(a.dist2) + i);
            if (a.b1_eqm) {  // Dist1 = 0 on B1 (a clear equal-q bit)
                const uint32_t ew = __ldg(reinterpret_cast<const uint32_t*>(a.b1_eqm) + i);
                if ((ew & 0x3Fu) != 0x3Fu) d1.x = 0;
                if (((ew >> 8) & 0x3Fu) != 0x3Fu) d1.y = 0;
                if (((ew >> 16) & 0x3Fu) != 0x3Fu) d1.z = 0;
                if (((ew >> 24) & 0x3Fu) != 0x3Fu) d1.w = 0;
            }
            float te, tp;
            grad_terms(g.x, (int8_t)(sw & 0xFF), d1.x, d2.x, a.p, te, tp);
            acc.add(te, tp);
            grad_terms(g.y, (int8_t)((sw >> 8) & 0xFF), d1.y, d2.y, a.p, te, tp);
            acc.add(te, tp);
            grad_terms(g.z, (int8_t)((sw >> 16) & 0xFF), d1.z, d2.z, a.p, te, tp);
            acc.add(te, tp);
            grad_terms(g.w, (int8_t)(sw >> 24), d1.w, d2.w, a.p, te, tp);
            acc.add(te, tp);
        }
    } else {
        for (int64_t i = t0; i < a.N; i += stride) {
            const int sv = __ldg(a.s + i);
            const float g = (sv || a.grad_dprime) ? __ldg(a.grad_out + i) : 0.f;
            if (a.grad_dprime) a.grad_dprime[i] = g;
            if (!sv) continue;
            int32_t d1 = __ldg(a.dist1 + i);
            if (a.b1_eqm && (__ldg(a.b1_eqm + i) & 0x3Fu) != 0x3Fu) d1 = 0;
            float te, tp;
            grad_terms(g, sv, d1, __ldg(a.dist2 + i), a.p, te, tp);
            acc.add(te, tp);
        }
    }
    acc.fold();
    double de = acc.de, dp = acc.dp;
    __shared__ double red[2][8];
    de = warp_sum(de);
    dp = warp_sum(dp);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = de;
        red[1][warp] = dp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double te = 0.0, tp = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            te += red[0][k];
            tp += red[1][k];
        }
        a.partials[2 * blockIdx.x] = te;
        a.partials[2 * blockIdx.x + 1] = tp;
    }
}

// Thread t adds partials t, t + 256, ... in order; thread 0 then adds the
// 256 subtotals in order. The order depends only on nblocks.
__global__ void __launch_bounds__(256) k_backward_final(BackArgs a, int nblocks)
{
    __shared__ double red[2][256];
    double te = 0.0, tp = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += 256) {
        te += a.partials[2 * k];
        tp += a.partials[2 * k + 1];
    }
    red[0][threadIdx.x] = te;
    red[1][threadIdx.x] = tp;
    __syncthreads();
    if (threadIdx.x != 0) return;
    te = tp = 0.0;
    for (int k = 0; k < 256; ++k) {
        te += red[0][k];
        tp += red[1][k];
    }
    a.grad_params[0] = te * a.eb;
    a.grad_params[1] = tp * a.eta * a.eb;
}

// The adjoint's saved state: S; Dist1 and Dist2 where S != 0 off B1, 0
// elsewhere (Dist2 was recorded into d2 at exactly those points). Four
// points per thread where N and the arrays allow.
__global__ void __launch_bounds__(256) k_save_signed(int64_t N, const int8_t* s, const uint8_t* eqm,
                                                      const int32_t* dist1, int8_t* s_out, int32_t* d1_out,
                                                      int32_t* d2, int vec)
{
    wait_prior_grid();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        for (int64_t i = t0; i < (N >> 2); i += stride) {
            const uint32_t sw = __ldg(reinterpret_cast<const uint32_t*>(s) + i);
            const uint32_t ew = __ldg(reinterpret_cast<const uint32_t*>(eqm) + i);
            reinterpret_cast<uint32_t*>(s_out)[i] = sw;
            unsigned keep = 0;  // bit j: S != 0 off B1
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (((sw >> (8 * j)) & 0xFFu) && ((ew >> (8 * j)) & 0x3Fu) == 0x3Fu) keep |= 1u << j;
            int4 o1 = make_int4(0, 0, 0, 0), o2 = make_int4(0, 0, 0, 0);
            if (keep) {
                const int4 a1 = __ldg(reinterpret_cast<const int4*>(dist1) + i);
                const int4 a2 = reinterpret_cast<const int4*>(d2)[i];
                o1 = make_int4(keep & 1u ? a1.x : 0, keep & 2u ? a1.y : 0, keep & 4u ? a1.z : 0, keep & 8u ? a1.w : 0);
                o2 = make_int4(keep & 1u ? a2.x : 0, keep & 2u ? a2.y : 0, keep & 4u ? a2.z : 0, keep & 8u ? a2.w : 0);
            }
            reinterpret_cast<int4*>(d1_out)[i] = o1;
            reinterpret_cast<int4*>(d2)[i] = o2;
        }
    } else {
        for (int64_t i = t0; i < N; i += stride) {
            const int sv = __ldg(s + i);
            s_out[i] = (int8_t)sv;
            const bool keep = sv && (__ldg(eqm + i) & 0x3Fu) == 0x3Fu;
            d1_out[i] = keep ? __ldg(dist1 + i) : 0;
            d2[i] = keep ? d2[i] : 0;
        }
    }
}

// The same from a plain forward's packed maps: S from spk (as int8), B1
// where the step-A code is not 0.
__global__ void __launch_bounds__(256) k_save_packed(int64_t N, const uint32_t* spk, const uint32_t* codes, int wpr,
                                                      int nx, const int32_t* dist1, int8_t* s_out, int32_t* d1_out,
                                                      int32_t* d2, int vec)
{
    wait_prior_grid();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        for (int64_t i = t0; i < (N >> 2); i += stride) {
            const unsigned sc = packed4(spk, wpr, nx, (int)(4 * i));
            uint32_t sw = 0;
            unsigned keep = 0;  // bit j: S != 0 off B1
            if (sc) {
                const unsigned cc = packed4(codes, wpr, nx, (int)(4 * i));
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int sv = s_of((sc >> (2 * j)) & 3u);
                    sw |= (uint32_t)(uint8_t)(int8_t)sv << (8 * j);
                    if (sv && !((cc >> (2 * j)) & 3u)) keep |= 1u << j;
                }
            }
            reinterpret_cast<uint32_t*>(s_out)[i] = sw;
            int4 o1 = make_int4(0, 0, 0, 0), o2 = make_int4(0, 0, 0, 0);
            if (keep) {
                const int4 a1 = __ldg(reinterpret_cast<const int4*>(dist1) + i);
                const int4 a2 = reinterpret_cast<const int4*>(d2)[i];
                o1 = make_int4(keep & 1u ? a1.x : 0, keep & 2u ? a1.y : 0, keep & 4u ? a1.z : 0, keep & 8u ? a1.w : 0);
                o2 = make_int4(keep & 1u ? a2.x : 0, keep & 2u ? a2.y : 0, keep & 4u ? a2.z : 0, keep & 8u ? a2.w : 0);
            }
            reinterpret_cast<int4*>(d1_out)[i] = o1;
            reinterpret_cast<int4*>(d2)[i] = o2;
        }
    } else {
        for (int64_t i = t0; i < N; i += stride) {
            const int sv = s_of(packed1(spk, wpr, nx, (int)i));
            s_out[i] = (int8_t)sv;
            const bool keep = sv && !packed1(codes, wpr, nx, (int)i);
            d1_out[i] = keep ? __ldg(dist1 + i) : 0;
            d2[i] = keep ? d2[i] : 0;
        }
    }
}

// D' = 2 q eps (Eq. 1) in fp32: float(q) * float(2 eps), rounded once, the
// expression every output of the library starts from.
__global__ void __launch_bounds__(256) k_dequantize(const int32_t* q, float* out, int64_t n, float two_eb)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = (float)__ldg(q + i) * two_eb;
}

// out = dprime + out: the last step of D'' = D' + C for a given D' (out
// holds C).
__global__ void __launch_bounds__(256) k_add_dprime(const float* dprime, float* out, int64_t n)
{
    wait_prior_grid();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = __ldg(dprime + i) + out[i];
}

int grid_for(int64_t n)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sms * 8));
}

}  // namespace

cudaError_t launch_dequantize(const int32_t* q, float* out, int64_t n, float two_eb, cudaStream_t st)
{
    k_dequantize<<<grid_for(n), 256, 0, st>>>(q, out, n, two_eb);
    return cudaGetLastError();
}

cudaError_t launch_add_dprime(const float* dprime, float* out, int64_t n, cudaStream_t st)
{
    return launch_chained(k_add_dprime, dim3(grid_for(n)), dim3(256), 0, st, dprime, out, n);
}

cudaError_t launch_save_packed(const LocalArgs& la, int8_t* s_out, int32_t* d1_out, int32_t* d2, cudaStream_t st)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto al = [](const void* p, int b) { return reinterpret_cast<uintptr_t>(p) % b == 0; };
    const int64_t N = (int64_t)la.nz * la.ny * la.nx;
    const int vec = la.nx % 4 == 0 && al(s_out, 4) && al(la.dist1, 16) && al(d1_out, 16) && al(d2, 16);
    return launch_chained(k_save_packed, dim3(sms * 8), dim3(256), 0, st, N, (const uint32_t*)la.spk,
                          (const uint32_t*)la.codes, la.wpr, la.nx, (const int32_t*)la.dist1, s_out, d1_out, d2, vec);
}

cudaError_t launch_save_signed(int64_t N, const int8_t* s, const uint8_t* eqm, const int32_t* dist1,
                               int8_t* s_out, int32_t* d1_out, int32_t* d2, cudaStream_t st)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto al = [](const void* p, int b) { return reinterpret_cast<uintptr_t>(p) % b == 0; };
    const int vec = N % 4 == 0 && al(s, 4) && al(eqm, 4) && al(s_out, 4) && al(dist1, 16) && al(d1_out, 16) && al(d2, 16);
    return launch_chained(k_save_signed, dim3(sms * 8), dim3(256), 0, st, N, s, eqm, dist1, s_out, d1_out, d2, vec);
}

cudaError_t launch_partials_sum(const double* partials, int nblocks, double eb, double eta,
                                double* grad_params, cudaStream_t st)
{
    BackArgs a{};
    a.partials = const_cast<double*>(partials);
    a.grad_params = grad_params;
    a.eb = eb;
    a.eta = eta;
    k_backward_final<<<1, 256, 0, st>>>(a, nblocks);
    return cudaGetLastError();
}

cudaError_t launch_backward(const BackArgs& a, cudaStream_t st)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (a.N + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    if (blocks > kBackwardMaxBlocks) blocks = kBackwardMaxBlocks;
    if (blocks < 1) blocks = 1;
    auto al = [](const void* p) { return p == nullptr || reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    const int vec = a.N % 4 == 0 && al(a.grad_out) && al(a.dist1) && al(a.dist2) && al(a.grad_dprime) &&
                    (a.spk ? a.nx % 4 == 0 : reinterpret_cast<uintptr_t>(a.s) % 4 == 0);
    k_backward<<<(int)blocks, 256, 0, st>>>(a, vec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_backward_final<<<1, 256, 0, st>>>(a, (int)blocks);
    return cudaGetLastError();
}

}  // namespace qai
