// qai_device.cuh -- encodings, argument blocks and device helpers shared by
// the qai CUDA kernels (row pass, column pass) and their host launchers.
//
// Pipeline of Algorithm 4 on a field of extents (nz, ny, nx), x contiguous:
//
//   row pass 1     step A (Algorithm 2) + first EDT pass along x on B1
//   column pass 1  EDT along y, then z (Algorithm 1), carrying the sign of
//                  the nearest boundary; the last pass writes Dist1 and S
//                  (step C's propagation, Algorithm 3, happens for free)
//   row pass 2     GetBoundary(S) -> B2 (Algorithm 3) + EDT pass along x
//   column pass 2  EDT along y, then z; the last pass fuses step E
//                  (IDW compensation) so Dist2 never reaches memory.
//
// Intermediate words (all-ones = "no site reached yet"):
//   xword  u16  phase 1: (d << 2) | sign code, d = |x - x_site| <= 16382
//               phase 2: d
//   yword  u32  phase 1: (g << 2) | sign code, g = dx^2 + dy^2 < 2^30
//               phase 2: g
// Sign code: 0 -> 0, 1 -> +1, 2 -> -1.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qai {

constexpr uint16_t kInf16 = 0xFFFFu;
constexpr uint32_t kInf32 = 0xFFFFFFFFu;
constexpr int32_t kDistInf = 0x7FFFFFFF;

__host__ __device__ inline int sign_code(int s) { return s > 0 ? 1 : (s < 0 ? 2 : 0); }
__host__ __device__ inline int sign_of_code(int c) { return c == 1 ? 1 : (c == 2 ? -1 : 0); }

struct MethodArgs {
    float two_eb;        // 2 eps, the dequantization step of Eq. 1
    float eta_eb;        // eta * eps, the boundary error magnitude of step E
    float idw_power;     // p of the inverse-distance weights
    int idw_is_one;      // p == 1 (the paper's weights): no powf
    int grad_threshold;  // Algorithm 2 fast-varying test, integer form
    int sign_rule;       // 0 SUM, 1 FIRST
    int b2_rule;         // 0 SAME_Q, 1 LITERAL
};

// Row pass: one warp per x-row; rows enumerated (z, y).
struct RowArgs {
    int rank, nz, ny, nx;
    const int32_t* q;        // phase 1 input; phase 2 final: D' source
    uint8_t* eqm;            // phase 1 writes, phase 2 reads: equal-q neighbour mask
    const int8_t* s_in;      // phase 2: propagated sign map S
    const int32_t* dist1_in; // phase 2 final (rank 1)
    uint16_t* xw;            // non-final output words
    int32_t* dist1;          // phase 1 final (rank 1)
    int8_t* s_out;           // phase 1 final (rank 1)
    float* out;              // phase 2 final (rank 1)
    // optional per-step outputs (NULL = skip)
    uint8_t* dbg_b1;
    int8_t* dbg_sb;
    int32_t* dbg_idx;        // phase 1: nearest-site linear index along the row
    uint8_t* dbg_b2;
    int32_t* dbg_dist2;      // phase 2 final (rank 1)
    MethodArgs m;
};

// Column pass over lines along one axis. Element (plane p, row r, column c)
// lives at p * plane_stride + r * row_stride + c for every array involved.
struct ColArgs {
    const void* in;          // xword (IN = 2) or yword (IN = 4) input
    int L;                   // line length (rows along the pass axis)
    int C;                   // columns per plane (contiguous)
    int P;                   // planes
    int64_t row_stride, plane_stride;
    int bands;               // B, rows are split in B bands of ceil(L / B)
    void* out_w;             // non-final output words (yword)
    int32_t* dist1;          // phase 1 final
    int8_t* s_out;           // phase 1 final
    float* out;              // phase 2 final
    const int32_t* q;        // phase 2 final
    const int32_t* dist1_in; // phase 2 final
    const int8_t* s_in;      // phase 2 final
    const int32_t* dbg_idx_in;   // phase 1: carried nearest-site index
    int32_t* dbg_idx_out;
    int32_t* dbg_dist2;      // phase 2 final
    MethodArgs m;
};

// Step E for one point: C = S * w * eta * eps with the inverse-distance weight
// w = k2^p / (k1^p + k2^p) of the distances k1 = sqrt(Dist1), k2 = sqrt(Dist2);
// a point on B1 gets w = 1 (this takes precedence), a point on B2 gets w = 0,
// and a field without B2 gives w = 1 (the limit k2 -> infinity).
__device__ __forceinline__ float compensate(int32_t q, int32_t d1, int32_t d2, int s,
                                            const MethodArgs& m)
{
    float c = 0.0f;
    if (s != 0) {
        float w;
        if (d1 == 0) {
            w = 1.0f;
        } else if (d2 == 0) {
            w = 0.0f;
        } else if (d2 == kDistInf) {
            w = 1.0f;
        } else {
            float k1 = sqrtf((float)d1), k2 = sqrtf((float)d2);
            if (m.idw_is_one) {
                w = k2 / (k1 + k2);
            } else {
                float a = powf(k1, m.idw_power), b = powf(k2, m.idw_power);
                w = b / (a + b);
            }
        }
        c = (float)s * w * m.eta_eb;
    }
    return fmaf((float)q, m.two_eb, c);
}

}  // namespace qai
