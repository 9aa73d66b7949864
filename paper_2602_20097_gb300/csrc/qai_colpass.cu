// qai_colpass.cu -- column kernels: the y and z passes of the exact EDT
// (Algorithm 1, Maurer's lower envelope of parabolas), banded for the GPU.
//
// A CTA owns W adjacent columns (lanes = columns, so every row access is
// coalesced) and all L rows of them. The tile of input words is staged in
// shared memory with cp.async vector copies; the L rows are cut into B bands,
// one thread per (column, band):
//   build   each thread runs Algorithm 1's envelope construction (the
//           RemoveEDT stack) over its band alone; the stack holds row numbers
//           h, the values g come from the staged tile;
//   merge   one thread per column splices the B band stacks into the column's
//           envelope. Splicing band k onto bands < k pops from the tail of the
//           envelope and from the head of band k only while band k has fewer
//           than two accepted entries: after that every triple is one band k
//           already checked;
//   query   each thread finds the envelope parabola of its first row (first
//           the band that holds it, then a binary search: the index of the
//           minimiser never decreases with the row), then walks its rows as
//           Algorithm 1's query loop does, moving on only when the next
//           parabola is strictly lower, so ties keep the earlier (smaller)
//           row -- the nearest site with the smallest linear index once the
//           passes run x, then y, then z.
// Phase 1 carries the sign code of the nearest boundary; its last pass writes
// Dist1 and S = S_B[I1] (Algorithm 3's propagation). Phase 2's last pass fuses
// step E: Dist2 goes straight into the compensation and never to memory.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "qai_device.cuh"
#include "qai_launch.h"

namespace qai {
namespace {

constexpr int kMaxBands = 32;

// CTAs of `kern` that fit on the device at once (at least one per SM).
template <class K>
unsigned resident_grid(K kern, dim3 block, size_t smem)
{
    int dev = 0, sms = 152, per = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, (int)(block.x * block.y * block.z), smem) !=
            cudaSuccess || per < 1)
        per = 1;
    return (unsigned)(sms * per);
}
constexpr int kScanMax = 24;   // outward-scan fast path: rows settled within 24 rows

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
// envelope of (g1, h1) and the new one (f, i): c g2 - b g1 - a f - a b c > 0
// with a = h2 - h1, b = i - h2, c = i - h1, written as
// c (g2 - f) - b (g1 - f) - (a b) c. NARROW: every term fits 32 bits (the
// host checks 2 L max(g) + L^3 < 2^31); otherwise 64-bit products.
template <bool NARROW>
__device__ __forceinline__ bool hidden(int g1, int g2, int f, int h1, int h2, int i)
{
    const int a = h2 - h1, b = i - h2, c = i - h1;
    if (NARROW) return c * (g2 - f) - b * (g1 - f) - (a * b) * c > 0;
    return (long long)c * (g2 - f) - (long long)b * (g1 - f) - (long long)(a * b) * c > 0;
}

__device__ __forceinline__ void cp_async(void* dst, const void* src, int bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    if (bytes == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
    else if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}

// Writes the result of one point: `val` is its squared distance, `w` the
// input word of the winning row (phase 1: carries the sign code), `src` the
// element index of that row in the same column (phase 1 index carry).
// Dist1 of point idx for step E (0 on B1 when the local first EDT left it
// unstored there).
__device__ __forceinline__ int32_t dist1_at(const ColArgs& a, int64_t idx)
{
    const int32_t d = __ldg(a.dist1_in + idx);
    if (!a.b1_eqm) return d;
    return (__ldg(a.b1_eqm + idx) & 0x3Fu) != 0x3Fu ? 0 : d;
}

// Points of the signed-point route collected by one CTA of the last pass of
// the first EDT before they go to the global lists: the queries (S != 0 off
// B1) and the B1 points with S != 0.
constexpr int kQueryBuf = 768;
constexpr int kSignedBuf = 512;
struct QueryBuf {
    Query* e;   // [kQueryBuf] in shared memory
    int* n;     // shared count (may pass kQueryBuf: the route then gives up)
    int32_t* se;// [kSignedBuf]
    int* sn;    // shared count (may pass kSignedBuf: that list is then incomplete)
    int* full;  // shared flag: the global query list is over its capacity
};

template <int PHASE, int IN, bool FINAL, bool DEBUG, bool GRAD, class Word>
__device__ __forceinline__ void emit_point(const ColArgs& a, int idx, int src, int val, Word w, bool valid,
                                           GradAcc& acc, int& any_sign, const QueryBuf& qb)
{
    if (PHASE == 1) {
        const int code = valid ? (int)(w & 3u) : 0;
        if (!FINAL) {
            static_cast<uint32_t*>(a.out_w)[idx] = valid ? ((uint32_t)val << 2) | (uint32_t)code : kInf32;
        } else {
            if (!a.qlist) {
                a.dist1[idx] = valid ? val : kDistInf;
            } else if (code != 0) {
                // signed-point route: Dist1 matters only where S != 0, and a
                // point off B1 there is a query of the second EDT
                a.dist1[idx] = val;
                if (val > 0) {
                    // once the global list is over its capacity the route
                    // hands the field over whatever the count: the CTA stops
                    // collecting (its flag, then the shared count it leaves)
                    if (*static_cast<volatile int*>(qb.full) == 0) {
                        const int k = atomicAdd(qb.n, 1);
                        if (k < kQueryBuf) {
                            qb.e[k] = Query{idx, (val << 2) | code};
                        } else {
                            // a full buffer spills to the global list; should
                            // the tile fall back to the envelope path, these
                            // entries are listed twice (the same query, the
                            // same output)
                            bool over = *static_cast<const volatile int*>(a.route_ctr + kCtrQueries) > a.qcap;
                            if (!over) {
                                const int g = atomicAdd(a.route_ctr + kCtrQueries, 1);
                                if (g < a.qcap) a.qlist[g] = Query{idx, (val << 2) | code};
                                else over = true;
                            }
                            if (over) *static_cast<volatile int*>(qb.full) = 1;
                        }
                    }
                } else {
                    const int k = atomicAdd(qb.sn, 1);
                    if (k < kSignedBuf) qb.se[k] = idx;
                }
            }
            a.s_out[idx] = (int8_t)sign_of_code(code);
            any_sign += sign_of_code(code) != 0;
        }
        if (DEBUG && a.dbg_idx_out) a.dbg_idx_out[idx] = valid ? a.dbg_idx_in[src] : -1;
    } else {
        const int32_t d = valid ? val : kDistInf;
        if (!FINAL) {
            static_cast<uint32_t*>(a.out_w)[idx] = valid ? (uint32_t)val : kInf32;
        } else if (GRAD) {
            float te, tp;
            grad_terms(__ldg(a.grad_out + idx), __ldg(a.s_in + idx), __ldg(a.dist1_in + idx), d,
                       a.m.idw_power, te, tp);
            acc.add(te, tp);
        } else {
            const int sv = __ldg(a.s_in + idx);
            // signed-point route: row pass 1 wrote every point with S = 0
            if (!a.route_ctr || sv != 0) {
                a.out[idx] = compensate(__ldg(a.q + idx), dist1_at(a, idx), d, sv, a.m);
                if (a.d2rec) a.d2rec[idx] = d;
            }
            if (DEBUG && a.dbg_dist2) a.dbg_dist2[idx] = d;
        }
    }
}

// One CTA of the column pass: tile `blk` of the lines described by `a`.
// GRAD (last phase-2 pass only): accumulate the adjoint terms of step E
// instead of writing D'', and store the CTA's two sums in a.partials.
template <int PHASE, int IN, bool FINAL, bool DEBUG, bool NARROW, bool GRAD = false>
__device__ __forceinline__ void colpass_tile(const ColArgs& a, const int blk)
{
    GradAcc acc;
    using Word = std::conditional_t<IN == 2, uint16_t, uint32_t>;
    constexpr Word kWInf = IN == 2 ? (Word)kInf16 : (Word)kInf32;
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = blockDim.x, B = blockDim.y;
    const int col = threadIdx.x, band = threadIdx.y;
    const int tid = band * W + col, nthr = W * B;
    const int L = a.L;
    Word* tile = reinterpret_cast<Word*>(smem);                       // [L][W] input words
    uint16_t* stk = reinterpret_cast<uint16_t*>(tile + (size_t)L * W);  // [L][W] band stacks (rows h)
    uint16_t* segA = stk + (size_t)L * W;                               // [B][W] kept range of each band
    uint16_t* segE = segA + B * W;                                      // [B][W]
    uint16_t* lstb = segE + B * W;                                      // [B][W] bands of the envelope, in order
    uint16_t* lmap = lstb + B * W;                                      // [B][W] band -> its position in lst
    uint16_t* nlst = lmap + B * W;                                      // [W] number of such bands

    const int tiles_per_plane = (a.C + W - 1) / W;
    const int p = blk / tiles_per_plane;
    const int c0 = (blk - p * tiles_per_plane) * W;
    const int pbase = p * a.plane_stride;
    const int RS = a.row_stride;
    const Word* in = static_cast<const Word*>(a.in);

    __shared__ int s_fail;      // the fast path below could not settle a row
    __shared__ int s_sign[32];  // phase 1 final: points with S != 0 per column (W <= 32)
    __shared__ int s_total;     // phase 2 final: points with S != 0 in the tile
    constexpr bool kQueries = PHASE == 1 && FINAL;
    __shared__ Query s_qbuf[kQueries ? kQueryBuf : 1];
    __shared__ int32_t s_sbuf[kQueries ? kSignedBuf : 1];
    __shared__ int s_qn, s_qbase, s_sn, s_sbase, s_qfull;
    const QueryBuf qb{s_qbuf, &s_qn, s_sbuf, &s_sn, &s_qfull};
    if (tid == 0) s_fail = s_total = s_qn = s_sn = s_qfull = 0;
    if (PHASE == 1 && FINAL && tid < W) s_sign[tid] = 0;
    int any_sign = 0;  // phase 1 final: this thread's points with S != 0

    // Phase 2 final: where S = 0, C = S w eta eps = 0 and D'' = D' whatever
    // Dist2 is; a tile whose columns all lack S != 0 only streams D'.
    if (PHASE == 2 && FINAL && !DEBUG && a.col_count_in != nullptr) {
        const int cc = c0 + col;
        const int cnt = band == 0 && cc < a.C ? (int)a.col_count_in[(int64_t)p * a.C + cc] : 0;
        if (__syncthreads_count(cnt > 0) == 0) {
            if (GRAD) {
                if (tid == 0) a.partials[2 * blk] = a.partials[2 * blk + 1] = 0.0;
                return;
            }
            if (a.route_ctr) return;  // row pass 1 wrote D' here
            const int Lb = (a.L + B - 1) / B;
            const int r0 = min(a.L, band * Lb), r1 = min(a.L, r0 + Lb);
            if (cc < a.C) {
                for (int r = r0; r < r1; ++r) {
                    const int idx = pbase + r * RS + cc;
                    a.out[idx] = a.m.output_c ? 0.0f : fmaf((float)__ldg(a.q + idx), a.m.two_eb, 0.0f);
                }
            }
            return;
        }
        if (cnt) atomicAdd(&s_total, cnt);
        __syncthreads();
    }
    // few points with S != 0 in the tile (at most one per two threads): the
    // last pass scans for Dist2 at them alone, reading the input words from
    // global memory, and stages the tile only if it falls back to the
    // envelope; otherwise every row takes the fast path below
    const bool sign_scan = PHASE == 2 && FINAL && !DEBUG && a.col_count_in != nullptr && 2 * s_total <= nthr;

    // ---- stage the tile ----------------------------------------------------
    auto stage = [&]() {
        const int cols = min(W, a.C - c0);
        const int vb = a.load_bytes;
        if (vb) {
            const int row_bytes = W * IN;
            const int cpr = row_bytes / vb, vcpr = cols * IN / vb;
            const char* gsrc = reinterpret_cast<const char*>(in + pbase + c0);
            for (int e = tid; e < L * cpr; e += nthr) {
                const int r = e / cpr, k = e - r * cpr;
                char* dst = reinterpret_cast<char*>(tile) + r * row_bytes + k * vb;
                if (k < vcpr) {
                    cp_async(dst, gsrc + (size_t)r * RS * IN + k * vb, vb);
                } else {
                    for (int b = 0; b < vb; b += 4) *reinterpret_cast<uint32_t*>(dst + b) = 0xFFFFFFFFu;
                }
            }
            asm volatile("cp.async.wait_all;\n" ::: "memory");
        } else {
            const int wshift = __ffs(W) - 1;
            for (int e = tid; e < L * W; e += nthr) {
                const int r = e >> wshift, c = e & (W - 1);
                tile[e] = c < cols ? in[pbase + r * RS + c0 + c] : kWInf;
            }
        }
        __syncthreads();
    };
    if (!sign_scan) stage();

    const int Lb = (L + B - 1) / B;
    const int r0 = min(L, band * Lb), r1 = min(L, r0 + Lb);
    const int c = c0 + col;
    const Word* tcol = tile + col;  // element (r, col) at tcol[r * W]
    auto gat = [&](int r) { return gval<PHASE, IN>(tcol[r * W]); };

    // ---- small-distance fast path ------------------------------------------
    // Row r's minimiser r' satisfies (r - r')^2 <= best value found so far, so
    // an outward scan r, r-1, r+1, r-2, r+2, ... can stop at the first k with
    // k^2 > best. Taking r - k on ties (<=) and r + k only when strictly lower
    // returns exactly Algorithm 1's answer (the smallest r' among equal minima).
    // The scan is tried first with k <= kScanMax: a row is settled when its
    // best is below (kScanMax + 1)^2, since no farther row can reach that. If
    // any row of the tile is not settled, the whole tile takes the envelope
    // path below, which rewrites every output of the tile (same rows per thread).
    //
    // The last pass of the second EDT needs Dist2 only where S != 0: elsewhere
    // C = S w eta eps = 0 and D'' = D'. Those rows are written directly; the
    // others (sparse where signs are) get their exact Dist2 from an outward
    // scan without the kScanMax limit (Dist2 carries no index, so ties do not
    // matter). A thread that would scan more than 4 rows per row of its band
    // (about what the envelope path costs it) sends the tile to the envelope
    // path instead.
    {
        volatile int* vfail = &s_fail;  // any thread of the tile failed: all stop
        if (sign_scan) {
          if constexpr (PHASE == 2 && FINAL && !DEBUG) {
            if (c < a.C) {
                int steps = 0;
                // rows in groups of four: their sign and index loads are issued
                // together, ahead of the branches that use them
                for (int rb = r0; rb < r1 && !*vfail; rb += 4) {
                    int sv[4], qv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int idx = pbase + (rb + u) * RS + c;
                        sv[u] = rb + u < r1 ? (int)__ldg(a.s_in + idx) : 0;
                        qv[u] = rb + u < r1 && !GRAD && !a.route_ctr ? __ldg(a.q + idx) : 0;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int r = rb + u;
                        if (r >= r1) break;
                        const int idx = pbase + r * RS + c;
                        if (sv[u] == 0) {
                            if (!GRAD && !a.route_ctr)
                                a.out[idx] = a.m.output_c ? 0.0f : fmaf((float)qv[u], a.m.two_eb, 0.0f);
                            continue;
                        }
                        const Word* gcol = in + pbase + c;  // row r' at gcol[r' * RS]
                        const Word w0 = __ldg(gcol + (int64_t)r * RS);
                        int best = w0 != kWInf ? gval<PHASE, IN>(w0) : 0x7FFFFFFF;
                        bool over = false;
                        for (int k = 1; k * k <= best && (r - k >= 0 || r + k < L); ++k) {
                            if (++steps > 4 * Lb) {
                                over = true;
                                break;
                            }
                            if (r - k >= 0) {
                                const Word w = __ldg(gcol + (int64_t)(r - k) * RS);
                                const int v = gval<PHASE, IN>(w) + k * k;
                                if (w != kWInf && v < best) best = v;
                            }
                            if (r + k < L) {
                                const Word w = __ldg(gcol + (int64_t)(r + k) * RS);
                                const int v = gval<PHASE, IN>(w) + k * k;
                                if (w != kWInf && v < best) best = v;
                            }
                        }
                        if (over) {
                            *vfail = 1;
                            break;
                        }
                        emit_point<PHASE, IN, FINAL, DEBUG, GRAD>(a, idx, 0, best, (Word)0, best != 0x7FFFFFFF,
                                                                  acc, any_sign, qb);
                    }
                }
            }
          }
        } else if (c < a.C) {
            for (int r = r0; r < r1 && !*vfail; ++r) {
                Word bw = tcol[r * W];
                int bh = bw != kWInf ? r : -1;
                int best = bw != kWInf ? gval<PHASE, IN>(bw) : 0x7FFFFFFF;
                for (int k = 1; k <= kScanMax && k * k <= best; ++k) {
                    if (r - k >= 0) {
                        const Word w = tcol[(r - k) * W];
                        const int v = gval<PHASE, IN>(w) + k * k;
                        if (w != kWInf && v <= best) { best = v; bh = r - k; bw = w; }
                    }
                    if (r + k < L) {
                        const Word w = tcol[(r + k) * W];
                        const int v = gval<PHASE, IN>(w) + k * k;
                        if (w != kWInf && v < best) { best = v; bh = r + k; bw = w; }
                    }
                }
                if (best >= (kScanMax + 1) * (kScanMax + 1)) {
                    *vfail = 1;
                    break;
                }
                emit_point<PHASE, IN, FINAL, DEBUG, GRAD>(a, pbase + r * RS + c, pbase + bh * RS + c, best, bw, true, acc, any_sign, qb);
            }
        }
        __syncthreads();
    }
    const bool use_envelope = s_fail != 0;  // CTA-uniform
    if (GRAD && use_envelope) acc = GradAcc();  // the envelope path redoes every row

    auto envelope_path = [&]() {
    if (kQueries && tid == 0) s_qn = s_sn = 0;  // the envelope path emits every point again
    // ---- build: Algorithm 1's envelope over this band ------------------------
    uint16_t* scol = stk + col;  // stack entry i of this column at scol[i * W]
    {
        // the three top entries live in registers (h2, g2 on top); after a pop
        // the load of the new third entry overlaps the next RemoveEDT test
        int n = 0, h0 = 0, g0 = 0, h1 = 0, g1 = 0, h2 = 0, g2 = 0;
        for (int r = r0; r < r1; ++r) {
            const Word w = tcol[r * W];
            if (w == kWInf) continue;
            const int f = gval<PHASE, IN>(w);
            while (n >= 2 && hidden<NARROW>(g1, g2, f, h1, h2, r)) {
                --n;
                h2 = h1;
                g2 = g1;
                h1 = h0;
                g1 = g0;
                if (n >= 3) {
                    h0 = scol[(r0 + n - 3) * W];
                    g0 = gat(h0);
                }
            }
            scol[(r0 + n) * W] = (uint16_t)r;
            h0 = h1;
            g0 = g1;
            h1 = h2;
            g1 = g2;
            h2 = r;
            g2 = f;
            ++n;
        }
        segA[band * W + col] = (uint16_t)r0;  // the band's stack: rows r0 .. r0 + n
        segE[band * W + col] = (uint16_t)(r0 + n);
    }
    __syncthreads();

    // ---- merge the band envelopes of each column, as a tree -----------------
    // Round j splices the envelopes of adjacent groups of 2^j bands, all pairs
    // at once: Maurer's stack construction continued with the right group's
    // entries pops the left group's tail and the right group's head, and
    // stops once two right entries stand (every later triple was already
    // checked inside the right group). A band keeps its surviving entries as
    // the range [segA, segE) of its stack. The result equals Algorithm 1's
    // envelope up to parabolas that only touch it at one point, which never
    // win a query (a neighbour with a smaller row ties there).
    for (int span = 1; span < B; span <<= 1) {
        if ((band & (2 * span - 1)) == 0 && band + span < B) {
            const int g0 = band, gm = band + span, g1 = min(B, band + 2 * span);
            auto A_ = [&](int k) { return (int)segA[k * W + col]; };
            auto E_ = [&](int k) { return (int)segE[k * W + col]; };
            // left group: last two entries e1 (band k1, pos p1) and e2 (k2, p2)
            int nleft = 0;
            for (int k = g0; k < gm; ++k) nleft += E_(k) - A_(k);
            int k1 = gm - 1;
            while (k1 >= g0 && A_(k1) == E_(k1)) --k1;
            int kr = gm;
            while (kr < g1 && A_(kr) == E_(kr)) ++kr;
            if (k1 >= g0 && kr < g1) {
                int p1 = E_(k1) - 1, k2 = k1, p2 = p1 - 1;
                if (p2 < A_(k2)) {
                    k2 = k1 - 1;
                    while (k2 >= g0 && A_(k2) == E_(k2)) --k2;
                    p2 = k2 >= g0 ? E_(k2) - 1 : 0;
                }
                int e1h = scol[p1 * W], e2h = nleft >= 2 ? scol[p2 * W] : 0;
                int e1g = gat(e1h), e2g = nleft >= 2 ? gat(e2h) : 0;
                // right group: candidates in order, from band kc position pc
                int kc = kr, pc = A_(kr);
                int acc = 0, bh = 0, bg = 0, bk = 0, bp = 0;  // first accepted right entry
                while (kc < g1 && acc < 2) {
                    const int fh = scol[pc * W], fg = gat(fh);
                    for (;;) {
                        if (acc == 1) {
                            if (nleft == 0 || !hidden<NARROW>(e1g, bg, fg, e1h, bh, fh)) break;
                            segA[bk * W + col] = (uint16_t)(bp + 1);  // pop the right entry
                            acc = 0;
                        } else {
                            if (nleft < 2 || !hidden<NARROW>(e2g, e1g, fg, e2h, e1h, fh)) break;
                            segE[k1 * W + col] = (uint16_t)p1;  // pop the left group's last entry
                            --nleft;
                            k1 = k2;
                            p1 = p2;
                            e1h = e2h;
                            e1g = e2g;
                            if (nleft >= 2) {
                                p2 = p1 - 1;
                                if (p2 < A_(k2)) {
                                    k2 = k2 - 1;
                                    while (k2 >= g0 && A_(k2) == E_(k2)) --k2;
                                    p2 = E_(k2) - 1;
                                }
                                e2h = scol[p2 * W];
                                e2g = gat(e2h);
                            }
                        }
                    }
                    if (acc == 0) { bh = fh; bg = fg; bk = kc; bp = pc; }
                    ++acc;
                    if (++pc >= E_(kc)) {
                        ++kc;
                        while (kc < g1 && A_(kc) == E_(kc)) ++kc;
                        if (kc < g1) pc = A_(kc);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (band == 0) {  // the envelope's bands, in order; each band's first entry in lst at or after it
        uint16_t* lst = lstb + col;
        int nl = 0;
        for (int k = 0; k < B; ++k) {
            lmap[k * W + col] = (uint16_t)nl;
            if (segA[k * W + col] != segE[k * W + col]) lst[(nl++) * W] = (uint16_t)k;
        }
        for (int k = B - 1; k >= 0 && lmap[k * W + col] >= nl; --k) lmap[k * W + col] = (uint16_t)(nl > 0 ? nl - 1 : 0);
        nlst[col] = (uint16_t)nl;
    }
    __syncthreads();

    // ---- query -------------------------------------------------------------
    // The envelope is the concatenation of the kept ranges of the bands
    // lst[0 .. nl), in order.
    if (c >= a.C || r0 >= r1) return;
    const uint16_t* lst = lstb + col;
    const int nl = nlst[col];
    if (nl == 0) {  // empty column: no site reaches it
        for (int r = r0; r < r1; ++r)
            emit_point<PHASE, IN, FINAL, DEBUG, GRAD>(a, pbase + r * RS + c, 0, 0, (Word)0, false, acc, any_sign, qb);
        return;
    }
    // envelope entry of row r0: the first entry that the next one does not
    // beat at r0 (the minimiser's index never decreases with the row). Start
    // at this band's first kept entry (or the last entry before it) and step
    // left or right; the entry is rarely more than a band away.
    int li = lmap[band * W + col];
    int k = lst[li * W];
    int pos = k >= band ? segA[k * W + col] : segE[k * W + col] - 1;
    auto val_at = [&](int ps, int r) {
        const int hh = scol[ps * W];
        return gat(hh) + (hh - r) * (hh - r);
    };
    auto next_of = [&](int l, int ps, int& ln, int& pn) {  // pn < 0: none
        ln = l;
        pn = ps + 1;
        if (pn >= segE[lst[l * W] * W + col]) pn = l + 1 < nl ? segA[lst[(++ln) * W] * W + col] : -1;
    };
    auto prev_of = [&](int l, int ps, int& lp, int& pp) {  // pp < 0: none
        lp = l;
        pp = ps - 1;
        if (pp < segA[lst[l * W] * W + col]) pp = l > 0 ? segE[lst[(--lp) * W] * W + col] - 1 : -1;
    };
    {
        int ln, pn;
        next_of(li, pos, ln, pn);
        if (pn >= 0 && val_at(pos, r0) > val_at(pn, r0)) {
            do {  // move right while the next entry is strictly lower
                li = ln;
                pos = pn;
                next_of(li, pos, ln, pn);
            } while (pn >= 0 && val_at(pos, r0) > val_at(pn, r0));
        } else {
            int lp, pp;
            prev_of(li, pos, lp, pp);
            while (pp >= 0 && !(val_at(pp, r0) > val_at(pos, r0))) {  // move left
                li = lp;
                pos = pp;
                prev_of(li, pos, lp, pp);
            }
        }
    }
    k = lst[li * W];
    int endk = segE[k * W + col];
    int h = scol[pos * W];
    Word w = tcol[h * W];
    int g = gval<PHASE, IN>(w);
    // next entry: (li_n, pos_n), pos_n < 0 when there is none
    int li_n = li, pos_n = pos + 1;
    if (pos_n >= endk) pos_n = li + 1 < nl ? segA[lst[(++li_n) * W] * W + col] : -1;
    int hn = pos_n >= 0 ? scol[pos_n * W] : 0;
    Word wn = pos_n >= 0 ? tcol[hn * W] : (Word)0;
    int gn = gval<PHASE, IN>(wn);

    // the last phase-2 pass loads step E's operands one row ahead, so their
    // latency overlaps the walk
    constexpr bool kFuseE = PHASE == 2 && FINAL;
    int idx = pbase + r0 * RS + c;
    int pq = 0, pd1 = 0, ps = 0;
    float pg = 0.f;
    if (kFuseE) {
        if (GRAD) pg = __ldg(a.grad_out + idx);
        else pq = __ldg(a.q + idx);
        pd1 = dist1_at(a, idx);
        ps = __ldg(a.s_in + idx);
    }
    for (int r = r0; r < r1; ++r) {
        int nq = 0, nd1 = 0, nsg = 0;
        float ng = 0.f;
        if (kFuseE && r + 1 < r1) {
            if (GRAD) ng = __ldg(a.grad_out + idx + RS);
            else nq = __ldg(a.q + idx + RS);
            nd1 = dist1_at(a, idx + RS);
            nsg = __ldg(a.s_in + idx + RS);
        }
        while (pos_n >= 0 && g + (h - r) * (h - r) > gn + (hn - r) * (hn - r)) {
            if (li_n != li) {
                li = li_n;
                endk = segE[lst[li * W] * W + col];
            }
            pos = pos_n;
            h = hn;
            w = wn;
            g = gn;
            pos_n = pos + 1;
            if (pos_n >= endk) pos_n = li + 1 < nl ? segA[lst[(++li_n) * W] * W + col] : -1;
            if (pos_n >= 0) {
                hn = scol[pos_n * W];
                wn = tcol[hn * W];
                gn = gval<PHASE, IN>(wn);
            }
        }
        const int val = g + (h - r) * (h - r);
        if (kFuseE) {
            if (GRAD) {
                float te, tp;
                grad_terms(pg, ps, pd1, val, a.m.idw_power, te, tp);
                acc.add(te, tp);
            } else {
                if (!a.route_ctr || ps != 0) {
                    a.out[idx] = compensate(pq, pd1, val, ps, a.m);
                    if (a.d2rec) a.d2rec[idx] = val;
                }
                if (DEBUG && a.dbg_dist2) a.dbg_dist2[idx] = val;
            }
            pq = nq;
            pg = ng;
            pd1 = nd1;
            ps = nsg;
        } else {
            emit_point<PHASE, IN, FINAL, DEBUG, GRAD>(a, idx, pbase + h * RS + c, val, w, true, acc, any_sign, qb);
        }
        idx += RS;
    }
    };  // envelope_path
    if (use_envelope) {
        if (sign_scan) stage();
        envelope_path();
    }

    if constexpr (PHASE == 1 && FINAL) {  // the columns' counts of S != 0
        if (any_sign) atomicAdd(&s_sign[col], any_sign);
        __syncthreads();
        if (band == 0 && c < a.C && a.col_count_out)
            a.col_count_out[(int64_t)p * a.C + c] = (uint16_t)min(s_sign[col], 65535);
        // the tile's points go to the global lists with one atomic each
        const int nq = min(s_qn, kQueryBuf), ns = s_sn;
        if (a.qlist && (nq > 0 || ns > 0)) {
            if (tid == 0) {
                s_qbase = s_sbase = -1;
                if (nq > 0) s_qbase = atomicAdd(a.route_ctr + kCtrQueries, nq);
                if (ns > kSignedBuf)
                    *static_cast<volatile int*>(a.route_ctr + kCtrSignedOver) = 1;
                else if (ns > 0)
                    s_sbase = atomicAdd(a.route_ctr + kCtrSigned, ns);
            }
            __syncthreads();
            const int qbase = s_qbase, sbase = s_sbase;
            if (qbase >= 0)
                for (int i = tid; i < nq && qbase + i < a.qcap; i += nthr) a.qlist[qbase + i] = s_qbuf[i];
            if (sbase >= 0)
                for (int i = tid; i < ns && sbase + i < a.scap; i += nthr) a.slist[sbase + i] = s_sbuf[i];
        }
    }

    if constexpr (GRAD) {  // the CTA's two sums: a fixed float-float tree over the threads
        __shared__ float red[4][512];
        red[0][tid] = acc.se;
        red[1][tid] = -acc.ce;
        red[2][tid] = acc.sp;
        red[3][tid] = -acc.cp;
        __syncthreads();
        for (int n = nthr; n > 1;) {
            const int h = (n + 1) >> 1;
            if (tid < n - h) {
                ff_add(red[0][tid], red[1][tid], red[0][tid + h], red[1][tid + h]);
                ff_add(red[2][tid], red[3][tid], red[2][tid + h], red[3][tid + h]);
            }
            __syncthreads();
            n = h;
        }
        if (tid == 0) {
            a.partials[2 * blk] = (double)red[0][0] + (double)red[1][0];
            a.partials[2 * blk + 1] = (double)red[2][0] + (double)red[3][0];
        }
    }}

// One tile per CTA, or (a gated launch: the passes behind the signed-point
// route and the local first EDT, which mostly find nothing to do) a resident
// grid that loops over the tiles.
template <int PHASE, int IN, bool FINAL, bool DEBUG, bool NARROW>
__device__ __forceinline__ void k_colpass_body(const ColArgs& a, const int bx, const int gx)
{
    wait_prior_grid();
    if (!a.gate) {
        colpass_tile<PHASE, IN, FINAL, DEBUG, NARROW>(a, bx);
        return;
    }
    if (*static_cast<const volatile int*>(a.gate) == 0) return;  // the flag is not set
    const int tiles = ((a.C + (int)blockDim.x - 1) / (int)blockDim.x) * a.P;
    for (int blk = bx; blk < tiles; blk += gx) {
        colpass_tile<PHASE, IN, FINAL, DEBUG, NARROW>(a, blk);
        __syncthreads();
    }
}

template <int PHASE, int IN, bool FINAL, bool DEBUG, bool NARROW>
__global__ void __launch_bounds__(512, IN == 2 ? 3 : 2) k_colpass(ColArgs a)
{
    k_colpass_body<PHASE, IN, FINAL, DEBUG, NARROW>(a, blockIdx.x, gridDim.x);
}


// The last phase-2 pass in adjoint mode (IN = 2: 2-D fields, 4: 3-D).
template <int IN, bool NARROW>
__global__ void __launch_bounds__(512, 2) k_colpass_grad(ColArgs a)
{
    colpass_tile<2, IN, true, false, NARROW, true>(a, blockIdx.x);
}

template <int PHASE, int IN, bool FINAL>
cudaError_t go(ColArgs& a, bool debug, bool narrow, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        dim3 g = grid;
        if (a.gate) g.x = std::min<unsigned>(g.x, resident_grid(kern, block, smem));
        return launch_chained(kern, g, block, smem, st, a);
    };
    if (debug) return narrow ? run(k_colpass<PHASE, IN, FINAL, true, true>)
                             : run(k_colpass<PHASE, IN, FINAL, true, false>);
    return narrow ? run(k_colpass<PHASE, IN, FINAL, false, true>)
                  : run(k_colpass<PHASE, IN, FINAL, false, false>);
}

}  // namespace

bool choose_colpass(int L, int in_bytes, ColConfig* cfg, bool first_edt_last_pass)
{
    // Passes over the x-pass words (in_bytes 2: the y passes) take tiles of 8
    // columns, the z passes 32 (measured on 2-D fronts of 1800-row columns
    // and on a 98 x 1200 x 1200 front: narrow tiles spread long columns over
    // more CTAs, the short z columns want wide rows); 32 rows per band.
    (void)first_edt_last_pass;
    const int w = in_bytes == 4 ? 32 : 8;
    return choose_colpass_with(L, in_bytes, 32, w, cfg);
}

bool choose_colpass_with(int L, int in_bytes, int rows_per_band, int max_w, ColConfig* cfg)
{
    int B = (L + rows_per_band - 1) / rows_per_band;
    B = B < 2 ? 2 : (B > kMaxBands ? kMaxBands : B);
    if (B > L) B = L < 1 ? 1 : L;
    const size_t budget = 200 * 1024;
    for (int W = max_w; W >= 4; W >>= 1) {
        if (W * B > 512) continue;  // the kernels' launch bound
        const size_t smem = (size_t)L * W * (in_bytes + 2) + (size_t)4 * B * W * 2 + (size_t)W * 2;
        if (smem <= budget) {
            cfg->W = W;
            cfg->B = B;
            cfg->smem = (smem + 15) & ~(size_t)15;
            return true;
        }
    }
    return false;
}

void prepare_colpass(ColArgs& a, int in_bytes, const ColConfig& cfg, int64_t max_g)
{
    a.bands = cfg.B;
    a.load_bytes = 0;
    for (int vb = 16; vb >= 4; vb >>= 1) {
        const bool ok = ((int64_t)a.row_stride * in_bytes) % vb == 0 &&
                        ((int64_t)a.plane_stride * in_bytes) % vb == 0 &&
                        ((int64_t)a.C * in_bytes) % vb == 0 && (cfg.W * in_bytes) % vb == 0 &&
                        (reinterpret_cast<uintptr_t>(a.in) % vb) == 0;
        if (ok) { a.load_bytes = vb; break; }
    }
    const int64_t L = a.L;
    a.narrow = 2 * L * max_g + L * L * L < (int64_t)0x7FFFFFFF;
}

int colpass_blocks(const ColArgs& a, int W) { return ((a.C + W - 1) / W) * a.P; }

cudaError_t launch_colpass(int phase, int in_bytes, bool final_pass, ColArgs& a, const ColConfig& cfg,
                           bool debug, int64_t max_g, cudaStream_t st)
{
    prepare_colpass(a, in_bytes, cfg, max_g);
    const bool narrow = a.narrow != 0;
    const dim3 grid(colpass_blocks(a, cfg.W)), block(cfg.W, cfg.B);
    if (phase == 1) {
        if (in_bytes == 2) return final_pass ? go<1, 2, true>(a, debug, narrow, grid, block, cfg.smem, st)
                                             : go<1, 2, false>(a, debug, narrow, grid, block, cfg.smem, st);
        return go<1, 4, true>(a, debug, narrow, grid, block, cfg.smem, st);
    }
    if (in_bytes == 2) return final_pass ? go<2, 2, true>(a, debug, narrow, grid, block, cfg.smem, st)
                                         : go<2, 2, false>(a, debug, narrow, grid, block, cfg.smem, st);
    return go<2, 4, true>(a, debug, narrow, grid, block, cfg.smem, st);
}

namespace {
template <int PHASE, int IN, bool FINAL, bool NARROW>
__global__ void __launch_bounds__(512, IN == 2 ? 3 : 2) k_colpass_group(const __grid_constant__ GroupQueue q)
{
    run_group<ColArgs>(q, [&](const ColArgs& a, int b, int n) { k_colpass_body<PHASE, IN, FINAL, false, NARROW>(a, b, n); });
}
}  // namespace

cudaError_t launch_group_colpass(const GroupQueue& q, int phase, int in_bytes, bool final_pass, bool narrow, int W,
                                 int B, size_t smem, cudaStream_t st)
{
    const dim3 block(W, B);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int grid = std::min(group_total(q), persistent_grid(kern, W * B, smem));
        if (grid < 1) return cudaSuccess;
        return launch_chained(kern, dim3(grid), block, smem, st, q);
    };
#define QAI_COLG(P, I, F) (narrow ? run(k_colpass_group<P, I, F, true>) : run(k_colpass_group<P, I, F, false>))
    if (phase == 1) {
        if (in_bytes == 2) return final_pass ? QAI_COLG(1, 2, true) : QAI_COLG(1, 2, false);
        return QAI_COLG(1, 4, true);
    }
    if (in_bytes == 2) return final_pass ? QAI_COLG(2, 2, true) : QAI_COLG(2, 2, false);
    return QAI_COLG(2, 4, true);
#undef QAI_COLG
}

}  // namespace qai

namespace qai {

cudaError_t launch_colpass_grad(int in_bytes, ColArgs& a, const ColConfig& cfg, int64_t max_g, cudaStream_t st)
{
    prepare_colpass(a, in_bytes, cfg, max_g);
    const dim3 grid(colpass_blocks(a, cfg.W)), block(cfg.W, cfg.B);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, block, cfg.smem, st>>>(a);
        return cudaGetLastError();
    };
    if (in_bytes == 2) return a.narrow ? run(k_colpass_grad<2, true>) : run(k_colpass_grad<2, false>);
    return a.narrow ? run(k_colpass_grad<4, true>) : run(k_colpass_grad<4, false>);
}

}  // namespace qai
