// qai_static.cu -- qai_mitigate_static: the whole method on a fixed scratch
// array that is part of the library, for callers that cannot allocate device
// memory (see include/qai.h). Nothing here allocates: the array is a
// file-scope __device__ variable, and its device address is looked up once
// per device.
#include <cstdio>
#include <mutex>

#include "qai.h"
#include "qai_launch.h"

namespace {

// Workspace of the largest accepted field: at most 12 bytes per point for
// the byte maps (the rank-3 layout: equal-q mask 1, Dist1 4, S 1, xwords 2,
// ywords 4), a uint16 count per column of the last column pass (at most one
// byte per point, since that pass has at least two rows), four packed maps of
// 2 bits a point (step-A codes, two equal-neighbour maps, S) and the B2
// bitmap (1 bit), each rounded up to whole words per row, the lists of the
// signed-point route (two of N / 32 + 1024 queries of 8 bytes (N / 128 +
// 1024 in 2-D), N / 256 +
// 1024 signed boundary points of 4 bytes, at most 65536 leftover queries at
// 12 bytes, N / 32 + 4096 B2 sites of 8 bytes) and the 256-byte alignment of
// its slices: at most 15 N + 0.71 MiB for every shape of at most N points
// with an x extent of 16 or more (the worst is an x extent of 17, whose
// packed rows are nearly half padding), inside 15 N + 1 MiB. Narrower x extents
// round more of each row up and can need more; such shapes are rejected when
// they do.
constexpr int64_t kMaxPoints = QAI_STATIC_MAX_POINTS;
constexpr size_t kScratchBytes = (size_t)15 * (size_t)kMaxPoints + ((size_t)1 << 20);

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device. In host code the name
// g_scratch is a host-side stand-in, never a device address. The first lookup
// on a device loads this file's module there (lazy module loading), which
// commits the array's memory on that device; a failure to load or to commit
// it is reported here, as QAI_ERR_CUDA.
qai_status scratch_address(void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        char msg[160];
        snprintf(msg, sizeof msg, "qai_mitigate_static: no usable current device (%s)",
                 cudaGetErrorString(e));
        qai::set_last_error(msg);
        return QAI_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            char msg[160];
            snprintf(msg, sizeof msg, "qai_mitigate_static: cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
            qai::set_last_error(msg);
            return QAI_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return QAI_OK;
}

}  // namespace

extern "C" qai_status qai_mitigate_static(const int32_t* d_q, float* d_out, int rank,
                                          const int64_t* dims, double eb, const qai_params* params,
                                          cudaStream_t stream)
{
    qai::set_last_error("");
    size_t need = 0;
    qai_status s = qai_workspace_size(rank, dims, 0, &need);  // validates rank and dims
    if (s != QAI_OK) return s;
    int64_t n = 1;
    for (int a = 0; a < rank; ++a) n *= dims[a];
    if (n > kMaxPoints) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "qai_mitigate_static: %lld points exceed the static scratch limit of %lld points",
                 (long long)n, (long long)kMaxPoints);
        qai::set_last_error(msg);
        return QAI_ERR_SHAPE;
    }
    if (need > kScratchBytes) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "qai_mitigate_static: this shape needs %zu bytes of workspace, more than the %zu bytes "
                 "of the static scratch array",
                 need, kScratchBytes);
        qai::set_last_error(msg);
        return QAI_ERR_SHAPE;
    }
    void* ws = nullptr;
    if ((s = scratch_address(&ws)) != QAI_OK) return s;
    return qai_mitigate(d_q, d_out, rank, dims, eb, params, ws, kScratchBytes, stream, nullptr);
}
