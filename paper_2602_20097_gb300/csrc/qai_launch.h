// qai_launch.h -- host-side launchers of the qai kernels (internal).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "qai.h"
#include "qai_device.cuh"

namespace qai {

// Launches of the plain path's kernels with programmatic stream
// serialization: the next kernel is scheduled while the previous one drains
// (every such kernel starts with wait_prior_grid()).
template <class... P, class... A>
cudaError_t launch_chained(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

// Row pass (qai_rowpass.cu): phase 1 = step A + EDT-x of B1,
// phase 2 = GetBoundary(S) + EDT-x of B2; final = the field is rank 1.
int rowpass_warps(int nx);
size_t rowpass_smem(int nx, int warps);
// debug: also write the per-step outputs named in `a`.
cudaError_t launch_rowpass(int phase, bool final_pass, const RowArgs& a, bool debug, cudaStream_t st);
// Sets a.vec (128-bit accesses usable) from the extents and pointers.
void prepare_rowpass(RowArgs& a);
cudaError_t launch_rowpass_grouped(int phase, bool final_pass, const RowTable& t, cudaStream_t st);

// Column pass (qai_colpass.cu): EDT along y or z. in_bytes = 2 for an xword
// input (the pass right after a row pass), 4 for a yword input.
struct ColConfig {
    int W;        // columns per CTA (power of two)
    int B;        // bands per column
    size_t smem;  // dynamic shared memory bytes
};
// first_edt_last_pass: the tile of the last pass of the first EDT.
bool choose_colpass(int L, int in_bytes, ColConfig* cfg, bool first_edt_last_pass = false);
bool choose_colpass_with(int L, int in_bytes, int rows_per_band, int max_w, ColConfig* cfg);
// Sets a.bands, a.load_bytes and a.narrow for a launch with `cfg`.
void prepare_colpass(ColArgs& a, int in_bytes, const ColConfig& cfg, int64_t max_g);
int colpass_blocks(const ColArgs& a, int W);
// The last phase-2 column pass in adjoint mode: a.grad_out, a.partials set,
// one pair of FP64 sums per CTA (colpass_blocks(a, cfg.W) CTAs).
cudaError_t launch_colpass_grad(int in_bytes, ColArgs& a, const ColConfig& cfg, int64_t max_g, cudaStream_t st);
// max_g bounds the squared distances carried by the input words; it decides
// whether RemoveEDT can run on 32-bit products.
cudaError_t launch_colpass(int phase, int in_bytes, bool final_pass, ColArgs& a,
                           const ColConfig& cfg, bool debug, int64_t max_g, cudaStream_t st);

// Signed-point route of the second EDT (qai_signed.cu): the B2 bitmap, the
// two shell phases at the queries, the list of B2 sites and the brute-force
// search; each kernel reads the route counters and does nothing when it is
// not needed.
cudaError_t launch_route_b2map(const RouteArgs& a, cudaStream_t st);
cudaError_t launch_route_query(const RouteArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_route_query_mid(const RouteArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_route_b2list(const RouteArgs& a, cudaStream_t st);
cudaError_t launch_route_brute(const RouteArgs& a, int blocks, bool sparse, cudaStream_t st);
cudaError_t launch_route_sparse_sites(const RouteArgs& a, cudaStream_t st);

// The local first EDT (qai_local.cu): step A with the pre-written output and
// the packed codes, then S (packed), Dist1 and the queries by a bounded
// nearest-site search; the byte maps of the separable passes (mode 1: when
// the dense second EDT runs, 2: always) and the packed S from the separable
// first EDT's int8 S map (gated: when that EDT ran as the fallback).
cudaError_t launch_local_detect(const LocalArgs& a, cudaStream_t st);
// Step A in z-slabs (the host-memory pipeline): whether the field takes the
// tiled fast path, one slab of it (planes zb .. zb + zn - 1, its neighbour
// planes already in place), and the exact pass behind all the slabs.
bool local_detect_slabs(const LocalArgs& a);
cudaError_t launch_local_detect_slab(const LocalArgs& a, int zb, int zn, cudaStream_t st);
cudaError_t launch_local_detect_exact(const LocalArgs& a, cudaStream_t st);
// Outputs that changed after step A, written straight into the caller's
// mapped host buffer: the queries' outputs, or every output when a pass that
// rewrites more ran (the exact step A, the separable first EDT, the dense
// second EDT).
cudaError_t launch_host_fixup(const LocalArgs& a, float* h_out_mapped, cudaStream_t st);
cudaError_t launch_local_near(const LocalArgs& a, cudaStream_t st);
cudaError_t launch_local_expand(const LocalArgs& a, int mode, cudaStream_t st);
cudaError_t launch_local_pack_s(const LocalArgs& a, bool gated, cudaStream_t st);

// Adjoint reduction of step E (qai_backward.cu).
cudaError_t launch_backward(const BackArgs& a, cudaStream_t st);
// The adjoint's saved state from a plain call's workspace: S; Dist1 and Dist2
// where S != 0 off B1 (Dist1 from dist1, Dist2 already recorded in d2), 0
// elsewhere.
cudaError_t launch_save_signed(int64_t N, const int8_t* s, const uint8_t* eqm, const int32_t* dist1,
                               int8_t* s_out, int32_t* d1_out, int32_t* d2, cudaStream_t st);
// The same from the packed maps of a plain forward (the local first EDT's
// arguments `la`: S from spk, B1 from the step-A codes).
cudaError_t launch_save_packed(const LocalArgs& la, int8_t* s_out, int32_t* d1_out, int32_t* d2, cudaStream_t st);
// D' = 2 q eps in fp32 (n points), and out = dprime + out (D'' for a given D').
cudaError_t launch_dequantize(const int32_t* q, float* out, int64_t n, float two_eb, cudaStream_t st);
cudaError_t launch_add_dprime(const float* dprime, float* out, int64_t n, cudaStream_t st);
// Adds the per-CTA partial sums of the fused adjoint pass in a fixed order.
cudaError_t launch_partials_sum(const double* partials, int nblocks, double eb, double eta,
                                double* grad_params, cudaStream_t st);

// CTAs of `kern` resident on the device at once (at least one per SM): the
// grid of a persistent grouped launch.
template <class K>
int persistent_grid(K kern, int threads, size_t smem)
{
    int dev = 0, sms = 152, per = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess || per < 1) per = 1;
    return sms * per;
}
inline int group_total(const GroupQueue& q)
{
    int t = 0;
    for (int f = 0; f < q.n; ++f) t += q.vb[f];
    return t;
}

// Persistent grouped launches (the batched form; see GroupQueue): q.args
// holds one argument struct per field, of the type the kernel takes; fields
// of both ranks (and load widths) share a launch, the body instance picked
// per work item. LocalArgs: step A (mode as k_detect's), the nearest-site
// search, the byte maps, the packed S.
cudaError_t launch_group_detect(const GroupQueue& q, int mode, cudaStream_t st);
cudaError_t launch_group_near(const GroupQueue& q, cudaStream_t st);
cudaError_t launch_group_expand(const GroupQueue& q, int mode, cudaStream_t st);
cudaError_t launch_group_pack_s(const GroupQueue& q, int gated, cudaStream_t st);
// RouteArgs: the signed-point route's kernels.
enum RouteKernel { kRouteB2Sparse, kRouteBruteSparse, kRouteB2Map, kRouteQuery, kRouteQueryMid, kRouteB2List,
                   kRouteBrute };
cudaError_t launch_group_route(RouteKernel k, const GroupQueue& q, cudaStream_t st);
// RowArgs (rank 2 and 3, non-final): warps per CTA and the largest x extent.
cudaError_t launch_group_rowpass(const GroupQueue& q, int phase, int warps, int max_nx, cudaStream_t st);
// ColArgs prepared for a (W, B) tile: every field of the launch shares W, B,
// the phase, the input words, finality and narrow arithmetic; smem covers the
// longest line.
cudaError_t launch_group_colpass(const GroupQueue& q, int phase, int in_bytes, bool final_pass, bool narrow, int W,
                                 int B, size_t smem, cudaStream_t st);

// Records `msg` as qai_last_error() of the calling host thread.
void set_last_error(const char* msg);

// Quality metrics (qai_quality.cu). The field is viewed as nz x ny x nx with
// window extents m* and strides s* per axis (1 on the axes a field lacks).
struct QualArgs {
    const float* x;
    const float* y;
    int nz, ny, nx;
    int mz, my, mx;
    int sz, sy, sx;
    int nwz, nwy, nwx;  // window counts
    int tz, gx, gy;     // windows per CTA along z, CTA grid along x and y
    int vec;            // 16-byte staging copies (set by launch_quality_ssim)
    qai_quality_out* result;
    double* partials;
    float* map;         // per-window SSIM or nullptr
};
void plan_quality(QualArgs& a, int sms);
int quality_ssim_blocks(const QualArgs& a);
size_t quality_smem(const QualArgs& a);
// min / max / MSE / PSNR: `blocks` block partials (3 doubles each) then one block.
cudaError_t launch_quality_stats(QualArgs& a, int64_t N, int blocks, cudaStream_t st);
// SSIM: quality_ssim_blocks(a) partials (1 double each) then one block.
cudaError_t launch_quality_ssim(QualArgs& a, cudaStream_t st);

}  // namespace qai
