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
// Row pitch of the record array: rows 2 apart (stride 2) land 16 banks apart.
constexpr int kXsPitch = 24;
constexpr float kC1 = 1e-4f, kC2 = 9e-4f;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

// ---- stage 1: min / max of x and sum of squared differences ---------------

// Per-thread accumulator of stage 1. The sum of squared differences is an
// fp32 compensated (Kahan) sum, converted to FP64 once per thread: its error
// is below 2 eps32 of the thread's sum for the few thousand terms a thread
// adds. (A periodic FP64 fold inside the loop would put FP64 instructions on
// every element once the compiler predicates it, and the FP64 pipe is narrow.)
struct StatAcc {
    float lo = INFINITY, hi = -INFINITY;
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float xv, float yv)
    {
        lo = fminf(lo, xv);
        hi = fmaxf(hi, xv);
        const float e = xv - yv;
        const float t = fmaf(e, e, -c), u = s + t;
        c = (u - s) - t;
        s = u;
    }
};

// vec: x and y 16-byte aligned and N a multiple of 4 (float4 loads, four
// pairs in flight per thread).
__global__ void __launch_bounds__(256) k_stats(QualArgs a, int64_t N, int vec)
{
    StatAcc acc;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        const float4* x4 = reinterpret_cast<const float4*>(a.x);
        const float4* y4 = reinterpret_cast<const float4*>(a.y);
        const int64_t n4 = N >> 2;
        int64_t i = t0;
        for (; i + 3 * nth < n4; i += 4 * nth) {
            float4 xv[4], yv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xv[u] = __ldg(x4 + i + u * nth);
                yv[u] = __ldg(y4 + i + u * nth);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc.add(xv[u].x, yv[u].x);
                acc.add(xv[u].y, yv[u].y);
                acc.add(xv[u].z, yv[u].z);
                acc.add(xv[u].w, yv[u].w);
            }
        }
        for (; i < n4; i += nth) {
            const float4 xv = __ldg(x4 + i), yv = __ldg(y4 + i);
            acc.add(xv.x, yv.x);
            acc.add(xv.y, yv.y);
            acc.add(xv.z, yv.z);
            acc.add(xv.w, yv.w);
        }
    } else {
        for (int64_t i = t0; i < N; i += nth) acc.add(__ldg(a.x + i), __ldg(a.y + i));
    }
    float lo = acc.lo, hi = acc.hi;
    double d = (double)acc.s - (double)acc.c;
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

__device__ __forceinline__ void cp_async4(float* dst, const float* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async16(float* dst, const float* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// Row pitch (floats) of a staged plane region: 16-byte aligned rows.
__host__ __device__ __forceinline__ int stage_pitch(int fx_max) { return (fx_max + 3) & ~3; }

// Merges K records laid out like merge() with K a compile-time count.
template <int K>
__device__ __forceinline__ Rec merge_k(const float* base, int step, int stride, float c)
{
    float v[5][K];
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int f = 0; f < 5; ++f) v[f][i] = base[i * step + f * stride];
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        sa += v[0][i];
        sb += v[1][i];
    }
    Rec r{sa * (1.0f / K), sb * (1.0f / K), 0.f, 0.f, 0.f};
    float da2 = 0.f, db2 = 0.f, dab = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const float da = v[0][i] - r.ma, db = v[1][i] - r.mb;
        r.va += v[2][i];
        r.vb += v[3][i];
        r.cab += v[4][i];
        da2 = fmaf(da, da, da2);
        db2 = fmaf(db, db, db2);
        dab = fmaf(da, db, dab);
    }
    r.va = fmaf(c, da2, r.va);
    r.vb = fmaf(c, db2, r.vb);
    r.cab = fmaf(c, dab, r.cab);
    return r;
}

// Two-pass statistics of one row segment of MX raw values (MX, SX compile
// time: 7 and 2 read as four 8-byte words per field), in normalised units.
template <int MX>
__device__ __forceinline__ Rec segment_fixed(const float* pa, const float* pb, float lo, float inv, float inv2)
{
    float va_[MX + 1], vb_[MX + 1];
#pragma unroll
    for (int k = 0; k < MX; k += 2) {
        const float2 ta = *reinterpret_cast<const float2*>(pa + k);
        const float2 tb = *reinterpret_cast<const float2*>(pb + k);
        va_[k] = ta.x;
        va_[k + 1] = ta.y;
        vb_[k] = tb.x;
        vb_[k + 1] = tb.y;
    }
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int k = 0; k < MX; ++k) {
        sa += va_[k];
        sb += vb_[k];
    }
    const float ma = sa * (1.0f / MX), mb = sb * (1.0f / MX);
    float va = 0.f, vb = 0.f, cab = 0.f;
#pragma unroll
    for (int k = 0; k < MX; ++k) {
        const float da = va_[k] - ma, db = vb_[k] - mb;
        va = fmaf(da, da, va);
        vb = fmaf(db, db, vb);
        cab = fmaf(da, db, cab);
    }
    return Rec{(ma - lo) * inv, (mb - lo) * inv, va * inv2, vb * inv2, cab * inv2};
}

__device__ __forceinline__ Rec segment_any(const float* pa, const float* pb, int mx, float lo, float inv, float inv2)
{
    float sa = 0.f, sb = 0.f;
    for (int k = 0; k < mx; ++k) {
        sa += pa[k];
        sb += pb[k];
    }
    const float ma = sa / (float)mx, mb = sb / (float)mx;
    float va = 0.f, vb = 0.f, cab = 0.f;
    for (int k = 0; k < mx; ++k) {
        const float da = pa[k] - ma, db = pb[k] - mb;
        va = fmaf(da, da, va);
        vb = fmaf(db, db, vb);
        cab = fmaf(da, db, cab);
    }
    return Rec{(ma - lo) * inv, (mb - lo) * inv, va * inv2, vb * inv2, cab * inv2};
}

// FIXED: the paper's window 7 with stride 2 on x and window extents MY, MZ
// (7 or 1) known at compile time; otherwise everything comes from `a`.
template <bool FIXED, int MY, int MZ>
__global__ void __launch_bounds__(kThreads, 3) k_ssim(QualArgs a)
{
    constexpr int MX = 7, SX = 2;
    extern __shared__ __align__(16) float qsm[];
    const int tid = threadIdx.x;
    const int mx = FIXED ? MX : a.mx, my = FIXED ? MY : a.my, mz = FIXED ? MZ : a.mz;
    const int sx = FIXED ? SX : a.sx;
    const int bx = blockIdx.x % a.gx;
    const int rest = blockIdx.x / a.gx;
    const int by = rest % a.gy, bz = rest / a.gy;
    const int wx0 = bx * kTX, wy0 = by * kTY, wz0 = bz * a.tz;
    const int wz1 = min(a.nwz, wz0 + a.tz);
    const int cnt_x = min(kTX, a.nwx - wx0), cnt_y = min(kTY, a.nwy - wy0);
    const int FX = sx * (cnt_x - 1) + mx, FY = a.sy * (cnt_y - 1) + my;
    const int FYmax = a.sy * (kTY - 1) + my, FXmax = sx * (kTX - 1) + mx;
    const int P = stage_pitch(FXmax);
    const int stage = FYmax * P;                  // floats of one field's plane region
    float* buf = qsm;                             // [2 planes][2 fields][FYmax][P] raw values
    float* xs = buf + 4 * stage;                  // [5][FYmax][kXsPitch] row-segment records
    float* ring = xs + 5 * FYmax * kXsPitch;      // [mz][5][kThreads] plane records per window
    const int xs_stride = FYmax * kXsPitch;

    const float lo = (float)a.result->x_min;
    const double range = a.result->x_max - a.result->x_min;
    const float inv = range > 0.0 ? (float)(1.0 / range) : 1.0f;
    const float inv2 = inv * inv;

    const int ty = tid >> 4, tx = tid & 15;       // this thread's window in the tile
    const bool mine = ty < cnt_y && tx < cnt_x;
    const int z_first = wz0 * a.sz, z_last = (wz1 - 1) * a.sz + mz - 1;
    const int64_t plane = (int64_t)a.ny * a.nx;
    const int64_t origin = (int64_t)(wy0 * a.sy) * a.nx + wx0 * sx;
    const float cx = (float)mx, cxy = (float)(mx * my);
    const int n = mx * my * mz;
    const float den = n > 1 ? (float)(n - 1) : 1.0f;
    // 16-byte copies when every row start is 16-byte aligned; the region is
    // then rounded up to whole float4s, which stay inside the row since nx
    // and the region's first column are multiples of 4.
    const bool vec = a.vec != 0;
    const int FX4 = (FX + 3) >> 2;
    float acc = 0.f, acc_c = 0.f;  // compensated sum of this thread's windows

    auto issue = [&](int z) {
        float* dA = buf + ((z - z_first) & 1) * 2 * stage;
        float* dB = dA + stage;
        const float* gA = a.x + z * plane + origin;
        const float* gB = a.y + z * plane + origin;
        if (vec && FX4 <= 16) {  // lanes 0..15 of a half-warp cover one row
            const int c = tx << 2;
            if (tx < FX4) {
                for (int r = ty; r < FY; r += kThreads / 16) {
                    const int64_t off = (int64_t)r * a.nx + c;
                    cp_async16(dA + r * P + c, gA + off);
                    cp_async16(dB + r * P + c, gB + off);
                }
            }
        } else if (vec) {
            for (int e = tid; e < FY * FX4; e += kThreads) {
                const int r = e / FX4, c = (e - r * FX4) << 2;
                const int64_t off = (int64_t)r * a.nx + c;
                cp_async16(dA + r * P + c, gA + off);
                cp_async16(dB + r * P + c, gB + off);
            }
        } else {
            for (int e = tid; e < FY * FX; e += kThreads) {
                const int r = e / FX, c = e - r * FX;
                const int64_t off = (int64_t)r * a.nx + c;
                cp_async4(dA + r * P + c, gA + off);
                cp_async4(dB + r * P + c, gB + off);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    issue(z_first);
    int slot = 0;
    for (int z = z_first; z <= z_last; ++z) {
        // the plane after this one streams in while this one is reduced; its
        // buffer was last read by the x pass two planes back, which every
        // thread finished before the barrier that closed that plane's x pass
        if (z < z_last) {
            issue(z + 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const float* tA = buf + ((z - z_first) & 1) * 2 * stage;
        const float* tB = tA + stage;
        // x pass: the record of every (row, window column) segment, two-pass
        // over the raw values and then mapped to normalised units (means
        // shifted and scaled, centred sums scaled by inv^2)
        if (tx < cnt_x) {
            for (int r = ty; r < FY; r += kThreads / 16) {
                const float* pa = tA + r * P + sx * tx;
                const float* pb = tB + r * P + sx * tx;
                Rec rec;
                if constexpr (FIXED) rec = segment_fixed<MX>(pa, pb, lo, inv, inv2);
                else rec = segment_any(pa, pb, mx, lo, inv, inv2);
                put(xs + r * kXsPitch + tx, xs_stride, rec);
            }
        }
        __syncthreads();
        if (mine) {
            const float* src = xs + (a.sy * ty) * kXsPitch + tx;
            Rec r;
            if constexpr (FIXED) r = merge_k<MY>(src, kXsPitch, xs_stride, cx);
            else r = merge(src, kXsPitch, xs_stride, my, cx);
            put(ring + slot * 5 * kThreads + tid, kThreads, r);
        }
        const int zs = z - mz + 1;  // first plane of the window that ends here
        if (mine && zs >= z_first && (zs - z_first) % a.sz == 0) {
            Rec w;
            if constexpr (FIXED) w = merge_k<MZ>(ring + tid, 5 * kThreads, kThreads, cxy);
            else w = merge(ring + tid, 5 * kThreads, kThreads, mz, cxy);
            const float va = w.va / den, vb = w.vb / den, cab = w.cab / den;
            const float s = ((2.f * w.ma * w.mb + kC1) * (2.f * cab + kC2)) /
                            ((w.ma * w.ma + w.mb * w.mb + kC1) * (va + vb + kC2));
            const float t = s - acc_c, u = acc + t;
            acc_c = (u - acc) - t;
            acc = u;
            if (a.map) {
                const int wz = zs / a.sz;
                a.map[((int64_t)wz * a.nwy + wy0 + ty) * a.nwx + wx0 + tx] = s;
            }
        }
        slot = slot + 1 == mz ? 0 : slot + 1;
    }
    // CTA sum in a fixed order
    const double total = warp_sum((double)acc - (double)acc_c);
    __shared__ double red[kThreads / 32];
    if ((tid & 31) == 0) red[tid >> 5] = total;
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
    const size_t fy = (size_t)a.sy * (kTY - 1) + a.my;
    const size_t pitch = (size_t)stage_pitch(a.sx * (kTX - 1) + a.mx);
    return 4 * (4 * fy * pitch + 5 * fy * kXsPitch + (size_t)a.mz * 5 * kThreads);
}

void plan_quality(QualArgs& a, int sms)
{
    a.gx = (a.nwx + kTX - 1) / kTX;
    a.gy = (a.nwy + kTY - 1) / kTY;
    int tz = 32;
    const int64_t base = (int64_t)a.gx * a.gy;
    while (tz > 4 && base * ((a.nwz + tz - 1) / tz) < 6LL * sms) tz >>= 1;
    a.tz = std::min(tz, a.nwz);
}

int quality_ssim_blocks(const QualArgs& a) { return a.gx * a.gy * ((a.nwz + a.tz - 1) / a.tz); }

cudaError_t launch_quality_stats(QualArgs& a, int64_t N, int blocks, cudaStream_t st)
{
    const int vec = (N % 4 == 0) && (reinterpret_cast<uintptr_t>(a.x) % 16 == 0) &&
                    (reinterpret_cast<uintptr_t>(a.y) % 16 == 0);
    k_stats<<<blocks, 256, 0, st>>>(a, N, vec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_stats_final<<<1, 256, 0, st>>>(a, blocks, N);
    return cudaGetLastError();
}

cudaError_t launch_quality_ssim(QualArgs& a, cudaStream_t st)
{
    a.vec = (a.nx % 4 == 0) && (reinterpret_cast<uintptr_t>(a.x) % 16 == 0) &&
            (reinterpret_cast<uintptr_t>(a.y) % 16 == 0);
    const size_t smem = quality_smem(a);
    const int blocks = quality_ssim_blocks(a);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        kern<<<blocks, kThreads, smem, st>>>(a);
        return cudaGetLastError();
    };
    // the paper's setting (window 7, stride 2) on full-size axes runs unrolled
    const bool fx = a.mx == 7 && a.sx == 2;
    const bool fy7 = a.my == 7 && a.sy == 2, fz7 = a.mz == 7 && a.sz == 2;
    const bool fy1 = a.my == 1 && a.ny == 1, fz1 = a.mz == 1 && a.nz == 1;
    cudaError_t e;
    if (fx && fy7 && fz7) e = run(k_ssim<true, 7, 7>);
    else if (fx && fy7 && fz1) e = run(k_ssim<true, 7, 1>);
    else if (fx && fy1 && fz1) e = run(k_ssim<true, 1, 1>);
    else e = run(k_ssim<false, 0, 0>);
    if (e != cudaSuccess) return e;
    const int64_t windows = (int64_t)a.nwx * a.nwy * a.nwz;
    k_ssim_final<<<1, 256, 0, st>>>(a, blocks, windows);
    return cudaGetLastError();
}

}  // namespace qai
