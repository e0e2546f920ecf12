// Volumes against a reference column that is not a vertex of the query field.
//
// Given the reference vertex's member column, every vertex of the grid is an
// independent problem (Sec. 3: R(p_ref, .) is computed vertex by vertex), so a
// grid split into z-slabs across GPUs needs one exchange per reference: the
// M-float column, sent by the GPU whose slab holds the reference vertex.  These
// entry points are the receiving side: the column is staged as a one-vertex
// field (its statistics by the same per-vertex kernel as a loaded field, hence
// bit-identical to the owner's), and the volume kernels run with it as the
// reference field and the local slab as the query field.  A slab volume is then
// bit-equal to the corresponding vertex range of the whole-grid call.
#include "ndf_internal.h"

namespace ndf {

__global__ void gather_column_kernel(const float* __restrict__ field, int64_t M, int64_t N,
                                     int64_t v, float* __restrict__ out) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x)
        out[m] = field[m * N + v];
}

// The context's one-vertex reference field, filled from `column` (M floats,
// host or device) with its statistics: from the kernel that a load of the whole
// field takes them from (the column sort up to 1024 members, which needs M more
// floats for the sorted copy), so that they are the same bits.
static ndf_status stage_column(ndf_ctx* ctx, const float* column, int64_t M, Field** out) {
    cudaError_t e = ctx->col_data.reserve(sizeof(float) * 2 * (size_t)M);
    if (e == cudaSuccess) e = ctx->col_stats.reserve(2 * sizeof(double) + sizeof(int));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reference column staging");
    e = cudaMemcpyAsync(ctx->col_data.ptr, column, sizeof(float) * (size_t)M, cudaMemcpyDefault,
                        ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reference column copy");
    Field& f = ctx->col_field;
    f.live = true;
    f.M = M;
    f.Z = f.Y = f.X = f.N = 1;
    f.data = ctx->col_data.as<float>();
    f.mean = ctx->col_stats.as<double>();
    f.inv_norm = ctx->col_stats.as<double>() + 1;
    int* nonfinite = reinterpret_cast<int*>(ctx->col_stats.as<double>() + 2);
    if (M <= kSortTileMaxM) {
        f.sorted = ctx->col_data.as<float>() + M;
        e = launch_sort_columns(ctx, f, 0, 1, ctx->stream, nullptr, nonfinite);
    } else {
        f.sorted = nullptr;
        e = launch_field_stats(ctx, f, 0, 1, nonfinite);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reference column statistics");
    *out = &f;
    return NDF_OK;
}

static ndf_status query_field(ndf_ctx* ctx, int field_id, Field** out) {
    if (field_id < 0 || field_id >= (int)ctx->fields.size())
        return fail(ctx, NDF_ERR_ARG, "field id out of range");
    Field& f = ctx->fields[field_id];
    if (!f.live) return fail(ctx, NDF_ERR_STATE, "field has been freed");
    *out = &f;
    return NDF_OK;
}

}  // namespace ndf

using namespace ndf;

extern "C" {

ndf_status ndf_field_column(ndf_ctx* ctx, int field_id, int64_t vertex, float* out) {
    if (!ctx) return NDF_ERR_ARG;
    Field* f;
    ndf_status st = query_field(ctx, field_id, &f);
    if (st != NDF_OK) return st;
    if (vertex < 0 || vertex >= f->N)
        return fail(ctx, NDF_ERR_ARG, "vertex %lld out of [0, %lld)", (long long)vertex,
                    (long long)f->N);
    cudaSetDevice(ctx->device);
    const size_t bytes = sizeof(float) * (size_t)f->M;
    void* dev_out;
    bool is_host;
    if ((st = resolve_out(ctx, out, bytes, &dev_out, &is_host)) != NDF_OK) return st;
    gather_column_kernel<<<(unsigned)((f->M + 255) / 256), 256, 0, ctx->stream>>>(
        f->data, f->M, f->N, vertex, static_cast<float*>(dev_out));
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "column gather");
    return finish_out(ctx, out, dev_out, bytes, is_host);
}

ndf_status ndf_pearson_column(ndf_ctx* ctx, const float* ref_column, int query_field_id,
                              float* out) {
    if (!ctx) return NDF_ERR_ARG;
    if (!ref_column) return fail(ctx, NDF_ERR_ARG, "null reference column");
    Field* qf;
    ndf_status st = query_field(ctx, query_field_id, &qf);
    if (st != NDF_OK) return st;
    cudaSetDevice(ctx->device);
    const size_t bytes = sizeof(float) * (size_t)qf->N;
    void* dev_out;
    bool is_host;
    if ((st = resolve_out(ctx, out, bytes, &dev_out, &is_host)) != NDF_OK) return st;
    Field* rf;
    if ((st = stage_column(ctx, ref_column, qf->M, &rf)) != NDF_OK) return st;
    cudaError_t e = launch_pearson(ctx, *rf, *qf, 0, static_cast<float*>(dev_out));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pearson launch");
    return finish_out(ctx, out, dev_out, bytes, is_host);
}

ndf_status ndf_mi_ksg_column(ndf_ctx* ctx, const float* ref_column, int query_field_id, int k,
                             float* out) {
    if (!ctx) return NDF_ERR_ARG;
    if (!ref_column) return fail(ctx, NDF_ERR_ARG, "null reference column");
    Field* qf;
    ndf_status st = query_field(ctx, query_field_id, &qf);
    if (st != NDF_OK) return st;
    if (k < 1 || k >= qf->M) return fail(ctx, NDF_ERR_ARG, "need 1 <= k < M (k=%d)", k);
    if (k > kKsgMaxK) return fail(ctx, NDF_ERR_ARG, "k=%d above the supported %d", k, kKsgMaxK);
    if (qf->M > kKsgMaxM)
        return fail(ctx, NDF_ERR_ARG, "M=%lld above the supported %d", (long long)qf->M, kKsgMaxM);
    cudaSetDevice(ctx->device);
    if ((st = ensure_psi_table(ctx, qf->M + 1)) != NDF_OK) return st;
    cudaError_t e = ensure_sorted_columns(ctx, *qf);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sorted columns");
    const size_t bytes = sizeof(float) * (size_t)qf->N;
    void* dev_out;
    bool is_host;
    if ((st = resolve_out(ctx, out, bytes, &dev_out, &is_host)) != NDF_OK) return st;
    Field* rf;
    if ((st = stage_column(ctx, ref_column, qf->M, &rf)) != NDF_OK) return st;
    e = launch_ksg(ctx, *rf, *qf, nullptr, 0, 1, k, 0, qf->N, static_cast<float*>(dev_out), 0,
                   ctx->ksg_algorithm != NDF_KSG_BRUTE, 1, ctx->ksg_tile, nullptr, nullptr, nullptr,
                   nullptr, ctx->count_evals ? ctx->evals.as<unsigned long long>() : nullptr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ksg launch");
    return finish_out(ctx, out, dev_out, bytes, is_host);
}

}  // extern "C"
