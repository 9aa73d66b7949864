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

// vec: N a multiple of 4 and every array aligned for 4-point accesses.
__global__ void __launch_bounds__(256) k_backward(BackArgs a, int vec)
{
    GradAcc acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        const int64_t n4 = a.N >> 2;
        for (int64_t i = t0; i < n4; i += stride) {
            const float4 g = __ldg(reinterpret_cast<const float4*>(a.grad_out) + i);
            const int4 d1 = __ldg(reinterpret_cast<const int4*>(a.dist1) + i);
            const int4 d2 = __ldg(reinterpret_cast<const int4*>(a.dist2) + i);
            const uint32_t sw = __ldg(reinterpret_cast<const uint32_t*>(a.s) + i);
            if (a.grad_dprime) reinterpret_cast<float4*>(a.grad_dprime)[i] = g;
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
            const float g = __ldg(a.grad_out + i);
            if (a.grad_dprime) a.grad_dprime[i] = g;
            float te, tp;
            grad_terms(g, __ldg(a.s + i), __ldg(a.dist1 + i), __ldg(a.dist2 + i), a.p, te, tp);
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

}  // namespace

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
                    reinterpret_cast<uintptr_t>(a.s) % 4 == 0;
    k_backward<<<(int)blocks, 256, 0, st>>>(a, vec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_backward_final<<<1, 256, 0, st>>>(a, (int)blocks);
    return cudaGetLastError();
}

}  // namespace qai
