// qai_colpass.cu -- column kernels: the y and z passes of the exact EDT
// (Algorithm 1, Maurer's lower envelope of parabolas), banded for the GPU.
//
// A CTA owns W adjacent columns (lanes = columns, so every row access is
// coalesced) and all L rows of them. The tile of input words is staged in
// shared memory; the L rows are cut into B bands, one thread per
// (column, band):
//   build   each thread runs Algorithm 1's envelope construction (the
//           RemoveEDT stack) over its band alone; the stack holds row numbers
//           h, the values g come from the staged tile;
//   merge   one thread per column splices the B band stacks into the column's
//           envelope. Splicing band k onto bands < k pops from the tail of the
//           envelope and from the head of band k only while band k has fewer
//           than two accepted entries: after that every triple is one band k
//           already checked;
//   query   each thread finds the envelope parabola of its first row by binary
//           search (the index of the minimiser never decreases with the row),
//           then walks its rows as Algorithm 1's query loop does, moving on
//           only when the next parabola is strictly lower, so ties keep the
//           earlier (smaller) row -- the nearest site with the smallest linear
//           index once the passes run x, then y, then z.
// Phase 1 carries the sign code of the nearest boundary; its last pass writes
// Dist1 and S = S_B[I1] (Algorithm 3's propagation). Phase 2's last pass fuses
// step E: Dist2 goes straight into the compensation and never to memory.
#include <type_traits>

#include "qai_device.cuh"
#include "qai_launch.h"

namespace qai {
namespace {

constexpr int kMaxBands = 16;

template <int PHASE, int IN>
__device__ __forceinline__ int gval(uint32_t w)
{
    if (PHASE == 1) {
        const int v = (int)(w >> 2);
        return IN == 2 ? v * v : v;
    }
    return IN == 2 ? (int)(w * w) : (int)w;
}

// RemoveEDT of Algorithm 1: parabola (g2, h2) lies strictly above the lower
// envelope of (g1, h1) and the new one (f, i), i.e. c g2 - b g1 - a f - a b c
// > 0 with a = h2 - h1, b = i - h2, c = i - h1, written as
// c (g2 - f) - b (g1 - f) - (a b) c with 32-bit operands, 64-bit products.
__device__ __forceinline__ bool hidden(int g1, int g2, int f, int h1, int h2, int i)
{
    const int a = h2 - h1, b = i - h2, c = i - h1;
    const long long v = (long long)c * (g2 - f) - (long long)b * (g1 - f) - (long long)(a * b) * c;
    return v > 0;
}

template <int PHASE, int IN, bool FINAL>
__global__ void __launch_bounds__(512) k_colpass(ColArgs a)
{
    using Word = std::conditional_t<IN == 2, uint16_t, uint32_t>;
    constexpr Word kWInf = IN == 2 ? (Word)kInf16 : (Word)kInf32;
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = blockDim.x, B = blockDim.y;
    const int col = threadIdx.x, band = threadIdx.y;
    const int tid = band * W + col, nthr = W * B;
    const int L = a.L;
    Word* tile = reinterpret_cast<Word*>(smem);                       // [L][W]
    uint16_t* stk = reinterpret_cast<uint16_t*>(tile + (size_t)L * W);  // [L][W]
    uint16_t* segA = stk + (size_t)L * W;                               // [B][W]
    uint16_t* segE = segA + B * W;                                      // [B][W]
    uint16_t* segO = segE + B * W;                                      // [B][W]
    uint16_t* nsum = segO + B * W;                                      // [W]

    const int tiles_per_plane = (a.C + W - 1) / W;
    const int p = blockIdx.x / tiles_per_plane;
    const int c0 = (blockIdx.x - p * tiles_per_plane) * W;
    const int64_t pbase = (int64_t)p * a.plane_stride;
    const int wshift = __ffs(W) - 1;
    const Word* in = static_cast<const Word*>(a.in);

    // ---- stage the tile ----------------------------------------------------
#pragma unroll 4
    for (int e = tid; e < L * W; e += nthr) {
        const int r = e >> wshift, c = c0 + (e & (W - 1));
        tile[e] = c < a.C ? in[pbase + (int64_t)r * a.row_stride + c] : kWInf;
    }
    __syncthreads();

    // ---- build: Algorithm 1's envelope over this band ------------------------
    const int Lb = (L + B - 1) / B;
    const int r0 = min(L, band * Lb), r1 = min(L, r0 + Lb);
    {
        int n = 0, h1 = 0, h2 = 0, g1 = 0, g2 = 0;
        for (int r = r0; r < r1; ++r) {
            const Word w = tile[r * W + col];
            if (w == kWInf) continue;
            const int f = gval<PHASE, IN>(w);
            while (n >= 2 && hidden(g1, g2, f, h1, h2, r)) {
                --n;
                h2 = h1;
                g2 = g1;
                if (n >= 2) {
                    h1 = stk[(r0 + n - 2) * W + col];
                    g1 = gval<PHASE, IN>(tile[h1 * W + col]);
                }
            }
            stk[(r0 + n) * W + col] = (uint16_t)r;
            h1 = h2;
            g1 = g2;
            h2 = r;
            g2 = f;
            ++n;
        }
        segE[band * W + col] = (uint16_t)n;  // count; the merge turns it into an end
    }
    __syncthreads();

    // ---- merge the band envelopes of each column --------------------------
    if (band == 0) {
        int lst[kMaxBands];
        int nl = 0, total = 0;
        auto entry_h = [&](int pos) { return (int)stk[pos * W + col]; };
        auto entry_g = [&](int h) { return gval<PHASE, IN>(tile[h * W + col]); };
        for (int k = 0; k < B; ++k) {
            const int kb = min(L, k * Lb);
            const int cnt = segE[k * W + col];
            int A = kb;
            const int E = kb + cnt;
            if (cnt == 0) {
                segA[k * W + col] = (uint16_t)kb;
                segE[k * W + col] = (uint16_t)kb;
                continue;
            }
            for (int cur = A; cur < E && cur - A < 2; ++cur) {
                const int hf = entry_h(cur), gf = entry_g(hf);
                for (;;) {
                    const int lenb = cur - A;
                    int ht1, ht2;
                    if (lenb == 1) {
                        if (nl == 0) break;
                        ht1 = entry_h(A);
                        ht2 = entry_h(segE[lst[nl - 1] * W + col] - 1);
                    } else {
                        if (total < 2) break;
                        const int kl = lst[nl - 1];
                        const int e = segE[kl * W + col], s = segA[kl * W + col];
                        ht1 = entry_h(e - 1);
                        ht2 = (e - s >= 2) ? entry_h(e - 2)
                                           : entry_h(segE[lst[nl - 2] * W + col] - 1);
                    }
                    if (!hidden(entry_g(ht2), entry_g(ht1), gf, ht2, ht1, hf)) break;
                    if (lenb == 1) {
                        A = cur;  // band k's only accepted entry is popped
                    } else {
                        const int kl = lst[nl - 1];
                        const int e = segE[kl * W + col] - 1;
                        segE[kl * W + col] = (uint16_t)e;
                        --total;
                        if (e == segA[kl * W + col]) --nl;
                    }
                }
            }
            segA[k * W + col] = (uint16_t)A;
            segE[k * W + col] = (uint16_t)E;
            lst[nl++] = k;
            total += E - A;
        }
        int off = 0;
        for (int k = 0; k < B; ++k) {
            segO[k * W + col] = (uint16_t)off;
            off += segE[k * W + col] - segA[k * W + col];
        }
        nsum[col] = (uint16_t)off;
    }
    __syncthreads();

    // ---- query -------------------------------------------------------------
    const int c = c0 + col;
    if (c >= a.C || r0 >= r1) return;
    const int ns = nsum[col];

    auto emit = [&](int r, int val, Word w, int h, bool valid) {
        const int64_t idx = pbase + (int64_t)r * a.row_stride + c;
        if (PHASE == 1) {
            const int code = valid ? (int)(w & 3u) : 0;
            if (!FINAL) {
                static_cast<uint32_t*>(a.out_w)[idx] = valid ? ((uint32_t)val << 2) | (uint32_t)code
                                                             : kInf32;
            } else {
                a.dist1[idx] = valid ? val : kDistInf;
                a.s_out[idx] = (int8_t)sign_of_code(code);
            }
            if (a.dbg_idx_out)
                a.dbg_idx_out[idx] =
                    valid ? a.dbg_idx_in[pbase + (int64_t)h * a.row_stride + c] : -1;
        } else {
            const int32_t d = valid ? val : kDistInf;
            if (!FINAL) {
                static_cast<uint32_t*>(a.out_w)[idx] = valid ? (uint32_t)val : kInf32;
            } else {
                a.out[idx] = compensate(a.q[idx], a.dist1_in[idx], d, a.s_in[idx], a.m);
                if (a.dbg_dist2) a.dbg_dist2[idx] = d;
            }
        }
    };

    if (ns == 0) {
        for (int r = r0; r < r1; ++r) emit(r, 0, 0, 0, false);
        return;
    }
    // global envelope position -> stack position
    auto locate = [&](int m, int* kout) {
        for (int k = 0; k < B; ++k) {
            const int o = segO[k * W + col];
            const int len = segE[k * W + col] - segA[k * W + col];
            if (m >= o && m < o + len) {
                *kout = k;
                return segA[k * W + col] + (m - o);
            }
        }
        *kout = 0;
        return 0;  // not reached for 0 <= m < ns
    };
    auto value = [&](int m, int r) {
        int k;
        const int h = stk[locate(m, &k) * W + col];
        return gval<PHASE, IN>(tile[h * W + col]) + (h - r) * (h - r);
    };
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (value(mid, r0) > value(mid + 1, r0)) lo = mid + 1;
        else hi = mid;
    }
    int m = lo, k;
    int pos = locate(m, &k);
    int h = stk[pos * W + col];
    Word w = tile[h * W + col];
    int g = gval<PHASE, IN>(w);
    for (int r = r0; r < r1; ++r) {
        while (m + 1 < ns) {
            int kn = k, pn = pos + 1;
            if (pn >= segE[k * W + col]) {
                do { ++kn; } while (kn < B - 1 && segE[kn * W + col] == segA[kn * W + col]);
                pn = segA[kn * W + col];
            }
            const int hn = stk[pn * W + col];
            const Word wn = tile[hn * W + col];
            const int gn = gval<PHASE, IN>(wn);
            if (g + (h - r) * (h - r) > gn + (hn - r) * (hn - r)) {
                ++m;
                k = kn;
                pos = pn;
                h = hn;
                w = wn;
                g = gn;
            } else {
                break;
            }
        }
        emit(r, g + (h - r) * (h - r), w, h, true);
    }
}

}  // namespace

bool choose_colpass(int L, int in_bytes, ColConfig* cfg)
{
    int B = (L + 47) / 48;
    B = B < 2 ? 2 : (B > kMaxBands ? kMaxBands : B);
    if (B > L) B = L < 1 ? 1 : L;
    const size_t budget = 200 * 1024;
    for (int W = 32; W >= 4; W >>= 1) {
        const size_t smem = (size_t)L * W * (in_bytes + 2) + (size_t)3 * B * W * 2 + (size_t)W * 2;
        if (smem <= budget) {
            cfg->W = W;
            cfg->B = B;
            cfg->smem = (smem + 15) & ~(size_t)15;
            return true;
        }
    }
    return false;
}

cudaError_t launch_colpass(int phase, int in_bytes, bool final_pass, ColArgs& a,
                           const ColConfig& cfg, cudaStream_t st)
{
    a.bands = cfg.B;
    const int tiles = ((a.C + cfg.W - 1) / cfg.W) * a.P;
    const dim3 grid(tiles), block(cfg.W, cfg.B);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)cfg.smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, block, cfg.smem, st>>>(a);
        return cudaGetLastError();
    };
    if (phase == 1) {
        if (in_bytes == 2) return final_pass ? go(k_colpass<1, 2, true>) : go(k_colpass<1, 2, false>);
        return go(k_colpass<1, 4, true>);
    }
    if (in_bytes == 2) return final_pass ? go(k_colpass<2, 2, true>) : go(k_colpass<2, 2, false>);
    return go(k_colpass<2, 4, true>);
}

}  // namespace qai
