// qai_shard.cu -- each process's device work in the sharded forms of
// Algorithm 4 (Section VII-B, distributed-memory parallelization): the row
// passes of both EDTs on an extended slab and the last pass along axis 0 on
// a band, from the separable pipeline's kernels. The processes' exchanges are
// host code; this file only validates, lays out the launch arguments and
// launches.
//
// Why the exact form reproduces the whole-field result: the separable EDT
// runs its passes along x, then y, then z, and each pass only needs whole
// lines along its own axis. The x (and y) passes of a slab's own planes see
// whole lines; after the all-to-all, a band holds whole lines along axis 0
// for the last pass. The words carried between the passes are the same ones
// the one-process pipeline carries, so the tie rule (smallest linear index)
// and every output bit are the same.
#include <cmath>
#include <cstdint>

#include "qai.h"
#include "qai_device.cuh"
#include "qai_host.h"
#include "qai_launch.h"

using namespace qai::host;

namespace {

constexpr int kMaxX = 16383, kMaxLine = 4096;

// Extents {n0, n1[, n2]} in the kernels' terms (rank 2: nz = 1).
struct Box {
    int rank, nz, ny, nx;
    int64_t N;
};

qai_status make_box(int rank, const int64_t* d, Box* b, const char* what)
{
    if (!d) return fail(QAI_ERR_INVALID_ARG, "%s is NULL", what);
    if (rank != 2 && rank != 3) return fail(QAI_ERR_SHAPE, "sharded calls take rank 2 or 3, not %d", rank);
    int64_t N = 1;
    for (int a = 0; a < rank; ++a) {
        const int64_t lim = a == rank - 1 ? kMaxX : kMaxLine;
        if (d[a] < 1 || d[a] > lim)
            return fail(QAI_ERR_SHAPE, "%s[%d] = %lld outside 1..%lld", what, a, (long long)d[a], (long long)lim);
        N *= d[a];
    }
    if (N >= (1LL << 31)) return fail(QAI_ERR_SHAPE, "%s: 2^31 points or more", what);
    b->rank = rank;
    b->N = N;
    b->nz = rank == 3 ? (int)d[0] : 1;
    b->ny = (int)d[rank - 2];
    b->nx = (int)d[rank - 1];
    return QAI_OK;
}

qai_status take_params(const qai_params* params, qai_params* p)
{
    if (params) *p = *params;
    else qai_default_params(p);
    return check_params(p);
}

size_t rows_ws(const Box& b) { return b.rank == 3 ? align256((size_t)b.N * 2) : 0; }

}  // namespace

extern "C" {

qai_status qai_shard_sizes(int rank, const int64_t* ext_dims, size_t* ws_bytes, int* word_bytes)
{
    qai::set_last_error("");
    Box b;
    qai_status s = make_box(rank, ext_dims, &b, "ext_dims");
    if (s != QAI_OK) return s;
    if (ws_bytes) *ws_bytes = rows_ws(b);
    if (word_bytes) *word_bytes = rank == 3 ? 4 : 2;
    return QAI_OK;
}

qai_status qai_shard_rows(int phase, int rank, const int64_t* ext_dims, const int32_t* d_q, const int8_t* d_s,
                          uint8_t* d_eqm, void* d_words, void* d_ws, size_t ws_bytes, const qai_params* params,
                          cudaStream_t stream)
{
    qai::set_last_error("");
    if (phase != 1 && phase != 2) return fail(QAI_ERR_INVALID_ARG, "phase must be 1 or 2");
    if (!d_q || !d_eqm || !d_words || (phase == 2 && !d_s))
        return fail(QAI_ERR_INVALID_ARG, "d_q, d_eqm, d_words (and d_s in phase 2) must be non-NULL");
    qai_params p;
    qai_status s = take_params(params, &p);
    if (s != QAI_OK) return s;
    Box b;
    if ((s = make_box(rank, ext_dims, &b, "ext_dims")) != QAI_OK) return s;
    const size_t need = rows_ws(b);
    if (need && (!d_ws || ws_bytes < need))
        return fail(QAI_ERR_INVALID_ARG, "workspace %zu bytes < %zu needed", d_ws ? ws_bytes : (size_t)0, need);
    const qai::MethodArgs m = method_args(&p, 1.0);  // the row passes use no eps

    // Step A or GetBoundary(S), and the EDT pass along x.
    qai::RowArgs r{};
    r.rank = rank;
    r.nz = b.nz; r.ny = b.ny; r.nx = b.nx;
    r.q = d_q; r.eqm = d_eqm; r.m = m;
    if (phase == 2) r.s_in = d_s;
    uint16_t* xw = rank == 2 ? static_cast<uint16_t*>(d_words) : static_cast<uint16_t*>(d_ws);
    r.xw = xw;
    const double N = (double)b.N;
    cudaError_t e = timed_call(phase == 1 ? "shard_rowpass1" : "shard_rowpass2", N * (phase == 1 ? 7.0 : 4.0),
                               stream, [&] { return qai::launch_rowpass(phase, false, r, false, stream); });
    if (e != cudaSuccess) return cuda_fail(e, "row pass");
    if (rank == 2) return QAI_OK;

    // The pass along y of every plane of the slab.
    qai::ColArgs c{};
    c.in = xw; c.L = b.ny; c.C = b.nx; c.P = b.nz;
    c.row_stride = b.nx; c.plane_stride = (int64_t)b.ny * b.nx; c.m = m;
    c.out_w = d_words;
    qai::ColConfig cfg;
    if (!qai::choose_colpass(c.L, 2, &cfg)) return fail(QAI_ERR_SHAPE, "line length %d does not fit", c.L);
    const int64_t gx = (int64_t)(b.nx - 1) * (b.nx - 1);
    e = timed_call(phase == 1 ? "shard_colpass1_y" : "shard_colpass2_y", N * 6.0, stream,
                   [&] { return qai::launch_colpass(phase, 2, false, c, cfg, false, gx, stream); });
    return e == cudaSuccess ? QAI_OK : cuda_fail(e, "column pass along y");
}

qai_status qai_shard_lines(int phase, int rank, const int64_t* band_dims, const int64_t* dims, const void* d_words,
                           const int32_t* d_q, int32_t* d_dist1, int8_t* d_s, uint16_t* d_count, float* d_out,
                           double eb, const qai_params* params, cudaStream_t stream)
{
    qai::set_last_error("");
    if (phase != 1 && phase != 2) return fail(QAI_ERR_INVALID_ARG, "phase must be 1 or 2");
    if (!d_words || !d_dist1 || !d_s || !d_count || (phase == 2 && (!d_q || !d_out)))
        return fail(QAI_ERR_INVALID_ARG, "d_words, d_dist1, d_s, d_count (and d_q, d_out in phase 2) must be non-NULL");
    if (phase == 2 && (!(eb > 0.0) || !std::isfinite(eb)))
        return fail(QAI_ERR_INVALID_ARG, "eb must be finite and > 0");
    qai_params p;
    qai_status s = take_params(params, &p);
    if (s != QAI_OK) return s;
    Box bb, fb;
    if ((s = make_box(rank, band_dims, &bb, "band_dims")) != QAI_OK) return s;
    if ((s = make_box(rank, dims, &fb, "dims")) != QAI_OK) return s;
    for (int a = 0; a < rank; ++a)
        if (band_dims[a] > dims[a]) return fail(QAI_ERR_SHAPE, "band_dims[%d] > dims[%d]", a, a);
    const int L = (int)band_dims[0];
    const int in_bytes = rank == 3 ? 4 : 2;
    // the largest squared distance the words carry: the passes before this one
    const int64_t gx = (int64_t)(fb.nx - 1) * (fb.nx - 1);
    const int64_t max_g = rank == 3 ? gx + (int64_t)(fb.ny - 1) * (fb.ny - 1) : gx;

    qai::ColArgs c{};
    c.in = d_words; c.L = L; c.C = (int)(bb.N / L); c.P = 1;
    c.row_stride = c.C; c.plane_stride = 0;
    c.m = method_args(&p, phase == 2 ? eb : 1.0);
    qai::ColConfig cfg;
    if (!qai::choose_colpass(L, in_bytes, &cfg, phase == 1)) return fail(QAI_ERR_SHAPE, "line length %d does not fit", L);
    const double N = (double)bb.N;
    cudaError_t e;
    if (phase == 1) {
        c.dist1 = d_dist1; c.s_out = d_s; c.col_count_out = d_count;
        e = timed_call("shard_colpass1_final", N * (in_bytes + 4 + 1), stream,
                       [&] { return qai::launch_colpass(1, in_bytes, true, c, cfg, false, max_g, stream); });
    } else {
        c.out = d_out; c.q = d_q; c.dist1_in = d_dist1; c.s_in = d_s; c.col_count_in = d_count;
        e = timed_call("shard_colpass2_final", N * (in_bytes + 4 + 1 + 4 + 4), stream,
                       [&] { return qai::launch_colpass(2, in_bytes, true, c, cfg, false, max_g, stream); });
    }
    return e == cudaSuccess ? QAI_OK : cuda_fail(e, "column pass along axis 0");
}

qai_status qai_shard_copy(void* d_dst, int64_t dst_pitch, const void* d_src, int64_t src_pitch, int64_t width,
                          int64_t height, cudaStream_t stream)
{
    qai::set_last_error("");
    if (width < 0 || height < 0) return fail(QAI_ERR_INVALID_ARG, "width and height must be >= 0");
    if (width == 0 || height == 0) return QAI_OK;
    if (!d_dst || !d_src) return fail(QAI_ERR_INVALID_ARG, "d_dst and d_src must be non-NULL");
    if (dst_pitch < width || src_pitch < width) return fail(QAI_ERR_INVALID_ARG, "pitches must be >= width");
    cudaError_t e = cudaMemcpy2DAsync(d_dst, (size_t)dst_pitch, d_src, (size_t)src_pitch, (size_t)width,
                                      (size_t)height, cudaMemcpyDeviceToDevice, stream);
    return e == cudaSuccess ? QAI_OK : cuda_fail(e, "strided copy");
}

}  // extern "C"
