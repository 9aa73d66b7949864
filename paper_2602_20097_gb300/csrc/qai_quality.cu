// qai_quality.cu -- the quality metrics of Sec. III-B on the GPU: PSNR (Eq. 4)
// and SSIM (Eq. 3) averaged over sliding windows.
//
// Readings: both fields are normalised by the original field's range before
// SSIM (v' = (v - min x) / range x, a constant original is only shifted); the
// sample variances and covariance divide the centred sums by n - 1; windows
// of m = min(window, extent) points start at 0, stride, 2 stride, ... on every
// axis while they fit, and the field's SSIM is the mean over all of them.
//
// Stage 1 (k_stats): one grid-stride pass over x and y: exact min and max of
// x, and sum (x - y)^2 in fp32 with compensation, folded into FP64. A one-block
// kernel combines the block partials in a fixed order and writes min, max,
// MSE and PSNR.
//
// Stage 2 (k_ssim): a CTA owns 16 x 16 windows in (y, x) and a run of window
// positions along z, and streams the z-planes of its region through shared
// memory. Per plane: an x pass turns every 1 x mx row segment into a record
// (two means, two centred sums of squares, one centred cross sum; two-pass
// over the segment), a y pass merges my records per window, and a ring keeps
// the last mz plane records of each window; when a window's last plane
// arrives its mz records are merged and Eq. 3 is evaluated. Records of equal
// count c merge without cancellation: the mean is the mean of the means, and
// each centred sum is the sum of the parts plus c times the centred sum of
// the part means. Block sums of the per-window SSIM are FP64 and are added in
// a fixed order by a one-block kernel.
#include <algorithm>
#include <cmath>

#include "qai_device.cuh"
#include "qai_launch.h"

namespace qai {
namespace {

constexpr int kTX = 16, kTY = 16, kThreads = kTX * kTY;
constexpr float kC1 = 1e-4f, kC2 = 9e-4f;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

// ---- stage 1: min / max of x and sum of squared differences ---------------

__global__ void __launch_bounds__(256) k_stats(QualArgs a, int64_t N)
{
    float lo = INFINITY, hi = -INFINITY;
    float s = 0.f, c = 0.f;
    double d = 0.0;
    int since = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const float xv = __ldg(a.x + i), yv = __ldg(a.y + i);
        lo = fminf(lo, xv);
        hi = fmaxf(hi, xv);
        const float e = xv - yv;
        const float t = e * e - c, u = s + t;  // compensated sum
        c = (u - s) - t;
        s = u;
        if (++since == 64) {
            d += (double)s - (double)c;
            s = c = 0.f;
            since = 0;
        }
    }
    d += (double)s - (double)c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_down_sync(0xFFFFFFFFu, lo, o));
        hi = fmaxf(hi, __shfl_down_sync(0xFFFFFFFFu, hi, o));
    }
    d = warp_sum(d);
    __shared__ float rlo[8], rhi[8];
    __shared__ double rs[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        rlo[warp] = lo;
        rhi[warp] = hi;
        rs[warp] = d;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            lo = fminf(lo, rlo[k]);
            hi = fmaxf(hi, rhi[k]);
            d += rs[k];
        }
        a.partials[3 * blockIdx.x] = lo;
        a.partials[3 * blockIdx.x + 1] = hi;
        a.partials[3 * blockIdx.x + 2] = d;
    }
}

__global__ void __launch_bounds__(256) k_stats_final(QualArgs a, int nblocks, int64_t N)
{
    __shared__ double rlo[256], rhi[256], rs[256];
    double lo = INFINITY, hi = -INFINITY, s = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += 256) {
        lo = fmin(lo, a.partials[3 * k]);
        hi = fmax(hi, a.partials[3 * k + 1]);
        s += a.partials[3 * k + 2];
    }
    rlo[threadIdx.x] = lo;
    rhi[threadIdx.x] = hi;
    rs[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int k = 1; k < 256; ++k) {
        lo = fmin(lo, rlo[k]);
        hi = fmax(hi, rhi[k]);
        s += rs[k];
    }
    const double mse = s / (double)N;
    qai_quality_out* r = a.result;
    r->x_min = lo;
    r->x_max = hi;
    r->mse = mse;
    // Eq. 4; identical fields give +inf, a constant original -inf
    r->psnr = mse == 0.0 ? INFINITY : (hi > lo ? 20.0 * log10((hi - lo) / sqrt(mse)) : -INFINITY);
}

// ---- stage 2: SSIM ------------------------------------------------------------

// A record: means of the two fields and centred sums over c points.
struct Rec {
    float ma, mb, va, vb, cab;
};

__device__ __forceinline__ void put(float* base, int stride, const Rec& r)
{
    base[0] = r.ma;
    base[stride] = r.mb;
    base[2 * stride] = r.va;
    base[3 * stride] = r.vb;
    base[4 * stride] = r.cab;
}

// Merges k records of c points each, read at base + i * step (fields
// `stride` apart): exact up to rounding, no cancellation.
__device__ __forceinline__ Rec merge(const float* base, int step, int stride, int k, float c)
{
    float sa = 0.f, sb = 0.f;
    for (int i = 0; i < k; ++i) {
        sa += base[i * step];
        sb += base[i * step + stride];
    }
    const float inv = 1.0f / (float)k;
    Rec r{sa * inv, sb * inv, 0.f, 0.f, 0.f};
    float da2 = 0.f, db2 = 0.f, dab = 0.f;
    for (int i = 0; i < k; ++i) {
        const float* p = base + i * step;
        const float da = p[0] - r.ma, db = p[stride] - r.mb;
        r.va += p[2 * stride];
        r.vb += p[3 * stride];
        r.cab += p[4 * stride];
        da2 = fmaf(da, da, da2);
        db2 = fmaf(db, db, db2);
        dab = fmaf(da, db, dab);
    }
    r.va = fmaf(c, da2, r.va);
    r.vb = fmaf(c, db2, r.vb);
    r.cab = fmaf(c, dab, r.cab);
    return r;
}

__global__ void __launch_bounds__(kThreads, 3) k_ssim(QualArgs a)
{
    extern __shared__ __align__(16) float qsm[];
    const int tid = threadIdx.x;
    const int bx = blockIdx.x % a.gx;
    const int rest = blockIdx.x / a.gx;
    const int by = rest % a.gy, bz = rest / a.gy;
    const int wx0 = bx * kTX, wy0 = by * kTY, wz0 = bz * a.tz;
    const int wz1 = min(a.nwz, wz0 + a.tz);
    const int cnt_x = min(kTX, a.nwx - wx0), cnt_y = min(kTY, a.nwy - wy0);
    const int FX = a.sx * (cnt_x - 1) + a.mx, FY = a.sy * (cnt_y - 1) + a.my;
    const int FYmax = a.sy * (kTY - 1) + a.my, FXmax = a.sx * (kTX - 1) + a.mx;
    float* tA = qsm;                              // [FY][FX] normalised x
    float* tB = tA + FYmax * FXmax;               // [FY][FX] normalised y
    float* xs = tB + FYmax * FXmax;               // [5][FYmax][kTX] row-segment records
    float* ring = xs + 5 * FYmax * kTX;           // [mz][5][kThreads] plane records per window
    const int xs_stride = FYmax * kTX;

    const float lo = (float)a.result->x_min;
    const double range = a.result->x_max - a.result->x_min;
    const float inv = range > 0.0 ? (float)(1.0 / range) : 1.0f;

    const int ty = tid / kTX, tx = tid - ty * kTX;
    const bool mine = ty < cnt_y && tx < cnt_x;
    const int z_first = wz0 * a.sz, z_last = (wz1 - 1) * a.sz + a.mz - 1;
    const int64_t plane = (int64_t)a.ny * a.nx;
    const int64_t origin = (int64_t)(wy0 * a.sy) * a.nx + wx0 * a.sx;
    const float cx = (float)a.mx, cxy = (float)(a.mx * a.my);
    const int n = a.mx * a.my * a.mz;
    const float den = n > 1 ? (float)(n - 1) : 1.0f;
    double acc = 0.0;

    for (int z = z_first; z <= z_last; ++z) {
        // normalised plane region
        const float* gx_ = a.x + z * plane + origin;
        const float* gy_ = a.y + z * plane + origin;
        for (int e = tid; e < FY * FX; e += kThreads) {
            const int r = e / FX, c = e - r * FX;
            const int64_t off = (int64_t)r * a.nx + c;
            tA[e] = (__ldg(gx_ + off) - lo) * inv;
            tB[e] = (__ldg(gy_ + off) - lo) * inv;
        }
        __syncthreads();
        // x pass: one record per (row, window column), two-pass over mx points
        for (int e = tid; e < FY * cnt_x; e += kThreads) {
            const int r = e / cnt_x, j = e - r * cnt_x;
            const float* pa = tA + r * FX + a.sx * j;
            const float* pb = tB + r * FX + a.sx * j;
            float sa = 0.f, sb = 0.f;
            for (int k = 0; k < a.mx; ++k) {
                sa += pa[k];
                sb += pb[k];
            }
            const float ma = sa / cx, mb = sb / cx;
            float va = 0.f, vb = 0.f, cab = 0.f;
            for (int k = 0; k < a.mx; ++k) {
                const float da = pa[k] - ma, db = pb[k] - mb;
                va = fmaf(da, da, va);
                vb = fmaf(db, db, vb);
                cab = fmaf(da, db, cab);
            }
            put(xs + r * kTX + j, xs_stride, Rec{ma, mb, va, vb, cab});
        }
        __syncthreads();
        const int slot = (z - z_first) % a.mz;
        if (mine) {
            const Rec r = merge(xs + (a.sy * ty) * kTX + tx, kTX, xs_stride, a.my, cx);
            put(ring + slot * 5 * kThreads + tid, kThreads, r);
        }
        const int zs = z - a.mz + 1;  // first plane of the window that ends here
        if (mine && zs >= z_first && (zs - z_first) % a.sz == 0) {
            const Rec w = merge(ring + tid, 5 * kThreads, kThreads, a.mz, cxy);
            const float va = w.va / den, vb = w.vb / den, cab = w.cab / den;
            const float s = ((2.f * w.ma * w.mb + kC1) * (2.f * cab + kC2)) /
                            ((w.ma * w.ma + w.mb * w.mb + kC1) * (va + vb + kC2));
            acc += (double)s;
            if (a.map) {
                const int wz = zs / a.sz;
                a.map[((int64_t)wz * a.nwy + wy0 + ty) * a.nwx + wx0 + tx] = s;
            }
        }
    }
    // CTA sum in a fixed order
    acc = warp_sum(acc);
    __shared__ double red[kThreads / 32];
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) t += red[k];
        a.partials[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(256) k_ssim_final(QualArgs a, int nblocks, int64_t windows)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += 256) s += a.partials[k];
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int k = 1; k < 256; ++k) s += red[k];
    a.result->ssim = s / (double)windows;
    a.result->windows = windows;
}

}  // namespace

size_t quality_smem(const QualArgs& a)
{
    const size_t fy = (size_t)a.sy * (kTY - 1) + a.my, fx = (size_t)a.sx * (kTX - 1) + a.mx;
    return 4 * (2 * fy * fx + 5 * fy * kTX + (size_t)a.mz * 5 * kThreads);
}

void plan_quality(QualArgs& a, int sms)
{
    a.gx = (a.nwx + kTX - 1) / kTX;
    a.gy = (a.nwy + kTY - 1) / kTY;
    int tz = 32;
    const int64_t base = (int64_t)a.gx * a.gy;
    while (tz > 4 && base * ((a.nwz + tz - 1) / tz) < 8LL * sms) tz >>= 1;
    a.tz = std::min(tz, a.nwz);
}

int quality_ssim_blocks(const QualArgs& a) { return a.gx * a.gy * ((a.nwz + a.tz - 1) / a.tz); }

cudaError_t launch_quality_stats(QualArgs& a, int64_t N, int blocks, cudaStream_t st)
{
    k_stats<<<blocks, 256, 0, st>>>(a, N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_stats_final<<<1, 256, 0, st>>>(a, blocks, N);
    return cudaGetLastError();
}

cudaError_t launch_quality_ssim(QualArgs& a, cudaStream_t st)
{
    const size_t smem = quality_smem(a);
    cudaError_t e = cudaFuncSetAttribute(k_ssim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int blocks = quality_ssim_blocks(a);
    k_ssim<<<blocks, kThreads, smem, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t windows = (int64_t)a.nwx * a.nwy * a.nwz;
    k_ssim_final<<<1, 256, 0, st>>>(a, blocks, windows);
    return cudaGetLastError();
}

}  // namespace qai
