// qai_launch.h -- host-side launchers of the qai kernels (internal).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "qai_device.cuh"

namespace qai {

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
bool choose_colpass(int L, int in_bytes, ColConfig* cfg);
bool choose_colpass_with(int L, int in_bytes, int rows_per_band, int max_w, ColConfig* cfg);
// Sets a.bands, a.load_bytes and a.narrow for a launch with `cfg`.
void prepare_colpass(ColArgs& a, int in_bytes, const ColConfig& cfg, int64_t max_g);
int colpass_blocks(const ColArgs& a, int W);
cudaError_t launch_colpass_grouped(int phase, int in_bytes, bool final_pass, const ColTable& t,
                                   const ColConfig& cfg, cudaStream_t st);
// max_g bounds the squared distances carried by the input words; it decides
// whether RemoveEDT can run on 32-bit products.
cudaError_t launch_colpass(int phase, int in_bytes, bool final_pass, ColArgs& a,
                           const ColConfig& cfg, bool debug, int64_t max_g, cudaStream_t st);

// Adjoint reduction of step E (qai_backward.cu).
cudaError_t launch_backward(const BackArgs& a, cudaStream_t st);

// Records `msg` as qai_last_error() of the calling host thread.
void set_last_error(const char* msg);

}  // namespace qai
