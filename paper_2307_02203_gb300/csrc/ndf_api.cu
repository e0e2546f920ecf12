// C-ABI entry points of libndf.so: context, ensembles, exact estimators.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <utility>
#include <vector>

#include "device_common.cuh"
#include "ndf_internal.h"

namespace ndf {

cudaError_t DevBuf::reserve(size_t need) {
    if (need <= bytes && ptr) return cudaSuccess;
    release();
    size_t n = need < 256 ? 256 : need;
    cudaError_t e = cudaMalloc(&ptr, n);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        return e;
    }
    bytes = n;
    return cudaSuccess;
}

void Field::free_all() {
    void* ps[] = {data, mean, inv_norm, z_tf32, z_hi, z_lo, sorted};
    for (void* q : ps)
        if (q) cudaFree(q);
    data = nullptr;
    mean = inv_norm = nullptr;
    z_tf32 = z_hi = z_lo = nullptr;
    sorted = nullptr;
    live = false;
}

// A wait that nothing completes: an mbarrier expecting one arrival that never
// comes.  The bounded wait gives up (about a second) and reports kDevTimeout.
__global__ void selftest_wait_kernel(unsigned* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) report(status, kDevTimeout);
}

cudaError_t ctx_alloc(ndf_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    for (size_t i = 0; i < ctx->cache.size(); ++i) {
        if (ctx->cache[i].bytes == bytes) {
            *p = ctx->cache[i].ptr;
            ctx->cache.erase(ctx->cache.begin() + (long)i);
            return cudaSuccess;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation && !ctx->cache.empty()) {
        cudaGetLastError();
        ctx_trim(ctx);
        e = cudaMalloc(p, bytes);
    }
    if (e != cudaSuccess) *p = nullptr;
    return e;
}

void ctx_release(ndf_ctx* ctx, void* p, size_t bytes) {
    if (!p) return;
    ctx->cache.push_back({p, bytes});
    while (ctx->cache.size() > kCacheEntries) {
        cudaFree(ctx->cache.front().ptr);
        ctx->cache.erase(ctx->cache.begin());
    }
}

void ctx_trim(ndf_ctx* ctx) {
    for (auto& c : ctx->cache) cudaFree(c.ptr);
    ctx->cache.clear();
}

void release_field(ndf_ctx* ctx, Field& f) {
    const size_t fb = sizeof(float) * (size_t)f.M * (size_t)f.N;
    const size_t sb = sizeof(double) * (size_t)f.N;
    ctx_release(ctx, f.data, fb);
    ctx_release(ctx, f.sorted, fb);
    ctx_release(ctx, f.mean, sb);
    ctx_release(ctx, f.inv_norm, sb);
    f.data = f.sorted = nullptr;
    f.mean = f.inv_norm = nullptr;
    f.free_all();  // the standardised copies
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

PtrKind pointer_kind(const void* p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PTR_HOST;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? PTR_DEVICE
                                                                                : PTR_HOST;
}

ndf_status fail(ndf_ctx* ctx, ndf_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return st;
}

ndf_status cuda_fail(ndf_ctx* ctx, cudaError_t e, const char* what) {
    ndf_status st = (e == cudaErrorMemoryAllocation) ? NDF_ERR_OOM : NDF_ERR_CUDA;
    return fail(ctx, st, "%s: %s", what, cudaGetErrorString(e));
}

ndf_status check_pair(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx,
                      const Field** rf, const Field** qf) {
    int nf = (int)ctx->fields.size();
    if (ref_field < 0 || ref_field >= nf || query_field < 0 || query_field >= nf)
        return fail(ctx, NDF_ERR_ARG, "field id out of range");
    const Field& a = ctx->fields[ref_field];
    const Field& b = ctx->fields[query_field];
    if (!a.live || !b.live) return fail(ctx, NDF_ERR_STATE, "field has been freed");
    if (a.M != b.M || a.Z != b.Z || a.Y != b.Y || a.X != b.X)
        return fail(ctx, NDF_ERR_ARG, "reference and query fields differ in shape");
    if (ref_idx < 0 || ref_idx >= a.N)
        return fail(ctx, NDF_ERR_ARG, "ref_idx %lld out of [0, %lld)", (long long)ref_idx,
                    (long long)a.N);
    *rf = &a;
    *qf = &b;
    return NDF_OK;
}

ndf_status resolve_out(ndf_ctx* ctx, void* out, size_t bytes, void** dev_out, bool* is_host) {
    if (!out) return fail(ctx, NDF_ERR_ARG, "null output pointer");
    if (pointer_kind(out) == PTR_DEVICE) {
        *dev_out = out;
        *is_host = false;
        return NDF_OK;
    }
    cudaError_t e = ctx->out_tmp.reserve(bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "output staging allocation");
    *dev_out = ctx->out_tmp.ptr;
    *is_host = true;
    return NDF_OK;
}

// Reads and clears the device status word; call only after the stream has drained.
ndf_status check_device_status(ndf_ctx* ctx) {
    unsigned st = 0;
    unsigned* d = ctx->flag.as<unsigned>() + 1;
    cudaError_t e = cudaMemcpy(&st, d, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device status read");
    if (st == 0) return NDF_OK;
    cudaMemset(d, 0, sizeof st);
    if (st & kDevTimeout) return fail(ctx, NDF_ERR_TIMEOUT, "a bounded device wait gave up");
    if (st & kDevBadInput)
        return fail(ctx, NDF_ERR_ARG, "a device-resident index was outside the field");
    return fail(ctx, NDF_ERR_CUDA, "device reported status 0x%x", st);
}

ndf_status finish_out(ndf_ctx* ctx, void* out, const void* dev_out, size_t bytes, bool is_host) {
    if (!is_host) return NDF_OK;
    cudaError_t e = cudaMemcpyAsync(out, dev_out, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy of the result to the host");
    return check_device_status(ctx);
}

// psi(n) at positive integers for the device table.  Shift n up to x >= 20 with
// psi(x) = psi(x + 1) - 1/x, then the asymptotic series
//   psi(x) ~ ln x - 1/(2x) - sum_j B_2j / (2j x^2j)
// (Abramowitz & Stegun 6.3.18) through the x^-12 term; truncation < 1e-17.
double digamma_int_host(int64_t n) {
    double x = (double)n, shift = 0.0;
    while (x < 20.0) {
        shift += 1.0 / x;
        x += 1.0;
    }
    double r = 1.0 / x, r2 = r * r;
    double series = r2 * (1.0 / 12 - r2 * (1.0 / 120 - r2 * (1.0 / 252 - r2 * (1.0 / 240 -
                    r2 * (1.0 / 132 - r2 * (691.0 / 32760))))));
    return log(x) - 0.5 * r - series - shift;
}

ndf_status ensure_psi_table(ndf_ctx* ctx, int64_t n_max) {
    if (ctx->psi_n > n_max) return NDF_OK;
    int64_t n = n_max + 1;
    std::vector<double> h((size_t)n, 0.0);
    for (int64_t i = 1; i < n; ++i) h[(size_t)i] = digamma_int_host(i);
    cudaError_t e = ctx->psi.reserve(sizeof(double) * (size_t)n);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->psi.ptr, h.data(), sizeof(double) * (size_t)n,
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "digamma table upload");
    ctx->psi_n = n;
    return NDF_OK;
}

}  // namespace ndf

using namespace ndf;

extern "C" {

const char* ndf_status_str(int status) {
    switch (status) {
        case NDF_OK: return "ok";
        case NDF_ERR_ARG: return "invalid argument";
        case NDF_ERR_OOM: return "out of memory";
        case NDF_ERR_CUDA: return "CUDA error";
        case NDF_ERR_TIMEOUT: return "device wait timed out";
        case NDF_ERR_STATE: return "invalid state";
        case NDF_ERR_IO: return "I/O error";
        default: return "unknown status";
    }
}

ndf_status ndf_create(ndf_ctx** out, int device, void* cuda_stream) {
    if (!out) return NDF_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return NDF_ERR_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return NDF_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3) return NDF_ERR_CUDA;  // built for sm_103a only
    if (cudaSetDevice(device) != cudaSuccess) return NDF_ERR_CUDA;
    ndf_ctx* c = new (std::nothrow) ndf_ctx();
    if (!c) return NDF_ERR_OOM;
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return NDF_ERR_CUDA;
        }
        c->stream = c->own_stream;
    }
    if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->copy_event, cudaEventDisableTiming) != cudaSuccess) {
        ndf_destroy(c);
        return NDF_ERR_CUDA;
    }
    if (c->flag.reserve(256) != cudaSuccess || cudaMemset(c->flag.ptr, 0, 256) != cudaSuccess) {
        ndf_destroy(c);
        return NDF_ERR_OOM;
    }
    *out = c;
    return NDF_OK;
}

void ndf_destroy(ndf_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto& f : ctx->fields) f.free_all();
    ctx_trim(ctx);
    ctx->stage_x.release();
    ctx->stage_perm.release();
    ctx->out_tmp.release();
    ctx->psi.release();
    ctx->dbg.release();
    ctx->flag.release();
    ctx->zr.release();
    ctx->refidx.release();
    ctx->evals.release();
    ctx->ksg_work.release();
    ctx->render_buf.release();
    ctx->col_data.release();
    ctx->col_stats.release();
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    if (ctx->copy_event) cudaEventDestroy(ctx->copy_event);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

const char* ndf_last_error(const ndf_ctx* ctx) {
    return ctx ? ctx->last_error.c_str() : "null context";
}

ndf_status ndf_set_stream(ndf_ctx* ctx, void* cuda_stream) {
    if (!ctx) return NDF_ERR_ARG;
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (!ctx->own_stream &&
            cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(ctx, NDF_ERR_CUDA, "stream creation failed");
        ctx->stream = ctx->own_stream;
    }
    return NDF_OK;
}

ndf_status ndf_synchronize(ndf_ctx* ctx) {
    if (!ctx) return NDF_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    return check_device_status(ctx);
}

uint64_t ndf_launch_count(const ndf_ctx* ctx) { return ctx ? ctx->launches : 0; }

int64_t ndf_index(int64_t x, int64_t y, int64_t z, int64_t X, int64_t Y, int64_t Z) {
    if (x < 0 || y < 0 || z < 0 || x >= X || y >= Y || z >= Z) return -1;
    return (z * Y + y) * X + x;
}

// The statistics of vertices [v0, v1) and, when wanted, their sorted columns: up to
// 1024 members one sort launch writes both (reading src when given, a device field
// that it also copies into f.data), above that the statistics kernel and the
// shared-memory sort read f.data.
static cudaError_t stats_and_sorts(ndf_ctx* ctx, const Field& f, int64_t v0, int64_t v1, bool want_sorted,
                                   const float* src, int* d_flag) {
    if (want_sorted && f.M <= kSortTileMaxM) return launch_sort_columns(ctx, f, v0, v1, ctx->stream, src, d_flag);
    if (src) return cudaErrorInvalidValue;
    cudaError_t e = launch_field_stats(ctx, f, v0, v1, d_flag);
    if (e == cudaSuccess && want_sorted) e = launch_sort_columns(ctx, f, v0, v1, ctx->stream);
    return e;
}

ndf_status ndf_load_ensemble(ndf_ctx* ctx, const float* field, int64_t M, int64_t Z, int64_t Y,
                             int64_t X, int* field_id_out) {
    if (!ctx) return NDF_ERR_ARG;
    if (!field || !field_id_out) return fail(ctx, NDF_ERR_ARG, "null pointer");
    if (M < 2 || Z < 1 || Y < 1 || X < 1)
        return fail(ctx, NDF_ERR_ARG, "need M >= 2 and a non-empty grid");
    int64_t N = Z * Y * X;
    if (N / X / Y != Z || M > (int64_t(1) << 40) / N)
        return fail(ctx, NDF_ERR_ARG, "field too large");
    cudaSetDevice(ctx->device);
    Field f;
    f.M = M; f.Z = Z; f.Y = Y; f.X = X; f.N = N;
    size_t bytes = sizeof(float) * (size_t)M * (size_t)N;
    const bool want_sorted = M <= kKsgMaxM;  // the KSG searches need it
    cudaError_t e = ctx_alloc(ctx, (void**)&f.data, bytes);
    if (e == cudaSuccess) e = ctx_alloc(ctx, (void**)&f.mean, sizeof(double) * (size_t)N);
    if (e == cudaSuccess) e = ctx_alloc(ctx, (void**)&f.inv_norm, sizeof(double) * (size_t)N);
    if (e == cudaSuccess && want_sorted) e = ctx_alloc(ctx, (void**)&f.sorted, bytes);
    if (e != cudaSuccess) {
        release_field(ctx, f);
        return cuda_fail(ctx, e, "field allocation");
    }
    cudaMemcpyKind kind = pointer_kind(field) == PTR_DEVICE ? cudaMemcpyDeviceToDevice
                                                            : cudaMemcpyHostToDevice;
    int* d_flag = ctx->flag.as<int>();
    // A host field is uploaded in vertex ranges on the copy stream; the statistics and
    // the column sort of each range run on the context's stream as soon as that range
    // has arrived.  The ranges double from the first (short, so the statistics start
    // early) up to 8x its length: a range is M strided rows, and longer rows copy closer
    // to the link's contiguous rate.  A device field needs no ranges (below).
    int64_t chunk = ((int64_t)(64 << 20) / M + 31) / 32 * 32;
    if (chunk < 1024) chunk = 1024;
    e = cudaMemsetAsync(d_flag, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess && kind == cudaMemcpyDeviceToDevice) {
        // A device-resident field needs no ranges: up to 1024 members one sort launch
        // reads it in place and writes the copy, the statistics and the sorted columns;
        // above that one contiguous copy comes first.
        const bool fused = want_sorted && M <= kSortTileMaxM;
        if (!fused) e = cudaMemcpyAsync(f.data, field, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e == cudaSuccess) e = stats_and_sorts(ctx, f, 0, N, want_sorted, fused ? field : nullptr, d_flag);
    } else {
        if (e == cudaSuccess) e = cudaEventRecord(ctx->copy_event, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_event, 0);
        int64_t len = chunk;
        for (int64_t v0 = 0; v0 < N && e == cudaSuccess; v0 += len, len = len * 2 < 8 * chunk ? len * 2 : 8 * chunk) {
            const int64_t v1 = v0 + len < N ? v0 + len : N;
            e = cudaMemcpy2DAsync(f.data + v0, sizeof(float) * (size_t)N, field + v0,
                                  sizeof(float) * (size_t)N, sizeof(float) * (size_t)(v1 - v0),
                                  (size_t)M, kind, ctx->copy_stream);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->copy_event, ctx->copy_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->copy_event, 0);
            if (e == cudaSuccess) e = stats_and_sorts(ctx, f, v0, v1, want_sorted, nullptr, d_flag);
        }
    }
    int nonfinite = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&nonfinite, d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess || nonfinite) {
        cudaStreamSynchronize(ctx->copy_stream);
        release_field(ctx, f);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "ensemble upload / statistics");
        return fail(ctx, NDF_ERR_ARG, "field contains non-finite values");
    }
    f.live = true;
    ctx->fields.push_back(f);
    *field_id_out = (int)ctx->fields.size() - 1;
    return NDF_OK;
}

// Upload, statistics, column sorts and the KSG search pipelined over vertex ranges:
// range r's search runs on the context's stream while range r + 1 is copied on the
// copy stream.  The reference's range goes first (both searches stage its column)
// and is short, so the search starts early; the rest of the grid follows in ranges
// that double up to 8x that length (a range is M strided rows, and longer rows copy
// closer to the link's contiguous rate; fewer ranges also mean fewer search launches).
ndf_status ndf_load_and_compute(ndf_ctx* ctx, const float* field, int64_t M, int64_t Z, int64_t Y,
                                int64_t X, int64_t ref_idx, int k, float* pearson_out,
                                float* mi_out, int* field_id_out) {
    if (!ctx) return NDF_ERR_ARG;
    if (!field || !field_id_out) return fail(ctx, NDF_ERR_ARG, "null pointer");
    if (M < 2 || Z < 1 || Y < 1 || X < 1)
        return fail(ctx, NDF_ERR_ARG, "need M >= 2 and a non-empty grid");
    const int64_t N = Z * Y * X;
    if (N / X / Y != Z || M > (int64_t(1) << 40) / N) return fail(ctx, NDF_ERR_ARG, "field too large");
    if (ref_idx < 0 || ref_idx >= N) return fail(ctx, NDF_ERR_ARG, "ref_idx out of range");
    if (mi_out) {
        if (k < 1 || k >= M) return fail(ctx, NDF_ERR_ARG, "need 1 <= k < M (k=%d)", k);
        if (k > kKsgMaxK) return fail(ctx, NDF_ERR_ARG, "k=%d above the supported %d", k, kKsgMaxK);
        if (M > kKsgMaxM) return fail(ctx, NDF_ERR_ARG, "M=%lld above the supported %d", (long long)M, kKsgMaxM);
    }
    cudaSetDevice(ctx->device);
    ndf_status st;
    if (mi_out && (st = ensure_psi_table(ctx, M + 1)) != NDF_OK) return st;
    Field f;
    f.M = M; f.Z = Z; f.Y = Y; f.X = X; f.N = N;
    const size_t bytes = sizeof(float) * (size_t)M * (size_t)N, vol = sizeof(float) * (size_t)N;
    // sorted as ndf_load_ensemble sorts (the KSG searches read the copy, and up to 1024
    // members the sort kernel writes the statistics), so the field left loaded, and the
    // Pearson volume from its statistics, are the same bits as after ndf_load_ensemble
    const bool want_sorted = M <= kKsgMaxM;
    cudaError_t e = ctx_alloc(ctx, (void**)&f.data, bytes);
    if (e == cudaSuccess) e = ctx_alloc(ctx, (void**)&f.mean, sizeof(double) * (size_t)N);
    if (e == cudaSuccess) e = ctx_alloc(ctx, (void**)&f.inv_norm, sizeof(double) * (size_t)N);
    if (e == cudaSuccess && want_sorted) e = ctx_alloc(ctx, (void**)&f.sorted, bytes);
    // outputs: device pointers as given, host ones staged in the context's scratch
    float *dp = nullptr, *dm = nullptr;
    const bool hp = pearson_out && pointer_kind(pearson_out) != PTR_DEVICE;
    const bool hm = mi_out && pointer_kind(mi_out) != PTR_DEVICE;
    if (e == cudaSuccess && (hp || hm)) e = ctx->out_tmp.reserve(2 * vol);
    if (e != cudaSuccess) {
        release_field(ctx, f);
        return cuda_fail(ctx, e, "allocation");
    }
    if (pearson_out) dp = hp ? ctx->out_tmp.as<float>() : pearson_out;
    if (mi_out) dm = hm ? ctx->out_tmp.as<float>() + N : mi_out;
    const cudaMemcpyKind kind = pointer_kind(field) == PTR_DEVICE ? cudaMemcpyDeviceToDevice
                                                                  : cudaMemcpyHostToDevice;
    int* d_flag = ctx->flag.as<int>();
    int64_t chunk = ((int64_t)(64 << 20) / M + 31) / 32 * 32;
    if (chunk < 1024) chunk = 1024;
    std::vector<std::pair<int64_t, int64_t>> ranges;
    {
        const int64_t r0 = ref_idx / chunk * chunk, r1 = r0 + chunk < N ? r0 + chunk : N;
        ranges.push_back({r0, r1});
        int64_t len = 2 * chunk;
        auto cover = [&](int64_t lo, int64_t hi) {
            for (int64_t v = lo; v < hi;) {
                const int64_t w = v + len < hi ? v + len : hi;
                ranges.push_back({v, w});
                v = w;
                len = len * 2 < 8 * chunk ? len * 2 : 8 * chunk;
            }
        };
        cover(r1, N);
        cover(0, r0);
    }
    // A device-resident field is not copied range by range: up to 1024 members each
    // range's sort launch reads the source and writes the copy as it goes; otherwise
    // one contiguous copy comes first.
    const bool dev = kind == cudaMemcpyDeviceToDevice;
    const bool dev_fused = dev && want_sorted && M <= kSortTileMaxM;
    e = cudaMemsetAsync(d_flag, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess && dev && !dev_fused)
        e = cudaMemcpyAsync(f.data, field, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->copy_event, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_event, 0);
    for (size_t q = 0; q < ranges.size() && e == cudaSuccess; ++q) {
        const int64_t v0 = ranges[q].first, v1 = ranges[q].second;
        if (!dev) {
            e = cudaMemcpy2DAsync(f.data + v0, sizeof(float) * (size_t)N, field + v0, sizeof(float) * (size_t)N,
                                  sizeof(float) * (size_t)(v1 - v0), (size_t)M, kind, ctx->copy_stream);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->copy_event, ctx->copy_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->copy_event, 0);
        }
        if (e == cudaSuccess)
            e = stats_and_sorts(ctx, f, v0, v1, want_sorted, dev_fused ? field : nullptr, d_flag);
        if (e == cudaSuccess && mi_out)
            e = launch_ksg(ctx, f, f, nullptr, ref_idx, 1, k, v0, v1, dm + v0, 0,
                           ctx->ksg_algorithm != NDF_KSG_BRUTE, 1, ctx->ksg_tile, nullptr, nullptr,
                           nullptr, nullptr,
                           ctx->count_evals ? ctx->evals.as<unsigned long long>() : nullptr);
    }
    if (e == cudaSuccess && pearson_out) e = launch_pearson(ctx, f, f, ref_idx, dp);
    int nonfinite = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&nonfinite, d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && hp) e = cudaMemcpyAsync(pearson_out, dp, vol, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && hm) e = cudaMemcpyAsync(mi_out, dm, vol, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess || nonfinite) {
        cudaStreamSynchronize(ctx->copy_stream);
        release_field(ctx, f);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "pipelined upload / volumes");
        return fail(ctx, NDF_ERR_ARG, "field contains non-finite values");
    }
    if ((st = check_device_status(ctx)) != NDF_OK) {
        release_field(ctx, f);
        return st;
    }
    f.live = true;
    ctx->fields.push_back(f);
    *field_id_out = (int)ctx->fields.size() - 1;
    return NDF_OK;
}

ndf_status ndf_free_ensemble(ndf_ctx* ctx, int field_id) {
    if (!ctx) return NDF_ERR_ARG;
    if (field_id < 0 || field_id >= (int)ctx->fields.size())
        return fail(ctx, NDF_ERR_ARG, "field id out of range");
    Field& f = ctx->fields[field_id];
    if (!f.live) return fail(ctx, NDF_ERR_STATE, "field already freed");
    cudaStreamSynchronize(ctx->stream);
    release_field(ctx, f);
    return NDF_OK;
}

ndf_status ndf_selftest_timeout(ndf_ctx* ctx) {
    if (!ctx) return NDF_ERR_ARG;
    cudaSetDevice(ctx->device);
    selftest_wait_kernel<<<1, 32, 0, ctx->stream>>>(ctx->flag.as<unsigned>() + 1);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "self-test launch");
    return check_device_status(ctx);
}

ndf_status ndf_trim_cache(ndf_ctx* ctx) {
    if (!ctx) return NDF_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx_trim(ctx);
    return NDF_OK;
}

ndf_status ndf_field_shape(const ndf_ctx* ctx, int field_id, int64_t* M, int64_t* Z, int64_t* Y,
                           int64_t* X) {
    if (!ctx || field_id < 0 || field_id >= (int)ctx->fields.size()) return NDF_ERR_ARG;
    const Field& f = ctx->fields[field_id];
    if (!f.live) return NDF_ERR_STATE;
    if (M) *M = f.M;
    if (Z) *Z = f.Z;
    if (Y) *Y = f.Y;
    if (X) *X = f.X;
    return NDF_OK;
}

ndf_status ndf_field_stats(ndf_ctx* ctx, int field_id, double* mean_out, double* inv_norm_out) {
    if (!ctx) return NDF_ERR_ARG;
    if (field_id < 0 || field_id >= (int)ctx->fields.size())
        return fail(ctx, NDF_ERR_ARG, "field id out of range");
    const Field& f = ctx->fields[field_id];
    if (!f.live) return fail(ctx, NDF_ERR_STATE, "field has been freed");
    size_t bytes = sizeof(double) * (size_t)f.N;
    cudaError_t e = cudaSuccess;
    if (mean_out) e = cudaMemcpyAsync(mean_out, f.mean, bytes, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess && inv_norm_out)
        e = cudaMemcpyAsync(inv_norm_out, f.inv_norm, bytes, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "statistics copy");
    return NDF_OK;
}

ndf_status ndf_field_sorted_columns(ndf_ctx* ctx, int field_id, int64_t v_begin, int64_t v_end,
                                    float* out) {
    if (!ctx) return NDF_ERR_ARG;
    if (field_id < 0 || field_id >= (int)ctx->fields.size())
        return fail(ctx, NDF_ERR_ARG, "field id out of range");
    Field& f = ctx->fields[field_id];
    if (!f.live) return fail(ctx, NDF_ERR_STATE, "field has been freed");
    if (v_begin < 0 || v_begin > v_end || v_end > f.N)
        return fail(ctx, NDF_ERR_ARG, "vertex range [%lld, %lld) outside [0, %lld)", (long long)v_begin,
                    (long long)v_end, (long long)f.N);
    if (f.M > kKsgMaxM) return fail(ctx, NDF_ERR_STATE, "no sorted columns above M = %d", kKsgMaxM);
    if (v_end == v_begin) return NDF_OK;
    if (!out) return fail(ctx, NDF_ERR_ARG, "null pointer");
    cudaSetDevice(ctx->device);
    cudaError_t e = ensure_sorted_columns(ctx, f);
    const size_t w = sizeof(float) * (size_t)(v_end - v_begin);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(out, w, f.sorted + v_begin, sizeof(float) * (size_t)f.N, w, (size_t)f.M,
                              cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sorted columns copy");
    return NDF_OK;
}

ndf_status ndf_pearson(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx, float* out) {
    if (!ctx) return NDF_ERR_ARG;
    const Field *rf, *qf;
    ndf_status st = check_pair(ctx, ref_field, query_field, ref_idx, &rf, &qf);
    if (st != NDF_OK) return st;
    cudaSetDevice(ctx->device);
    size_t bytes = sizeof(float) * (size_t)qf->N;
    void* dev_out;
    bool is_host;
    if ((st = resolve_out(ctx, out, bytes, &dev_out, &is_host)) != NDF_OK) return st;
    cudaError_t e = launch_pearson(ctx, *rf, *qf, ref_idx, (float*)dev_out);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pearson launch");
    return finish_out(ctx, out, dev_out, bytes, is_host);
}

static ndf_status check_ksg_args(ndf_ctx* ctx, const Field* rf, int k) {
    if (k < 1 || k >= rf->M) return fail(ctx, NDF_ERR_ARG, "need 1 <= k < M (k=%d)", k);
    if (k > kKsgMaxK) return fail(ctx, NDF_ERR_ARG, "k=%d above the supported %d", k, kKsgMaxK);
    if (rf->M > kKsgMaxM)
        return fail(ctx, NDF_ERR_ARG, "M=%lld above the supported %d", (long long)rf->M, kKsgMaxM);
    return NDF_OK;
}

// one reference over [v_begin, v_end) with the context's algorithm
static cudaError_t run_ksg_one(ndf_ctx* ctx, const Field& rf, const Field& qf, int64_t ref_idx,
                               int k, int64_t v_begin, int64_t v_end, float* out, double* dbg_mi,
                               float* dbg_eps, int32_t* dbg_nx, int32_t* dbg_ny, int variant = 1,
                               float* dbg_ey = nullptr) {
    return launch_ksg(ctx, rf, qf, nullptr, ref_idx, 1, k, v_begin, v_end, out, 0,
                      ctx->ksg_algorithm != NDF_KSG_BRUTE, 1, ctx->ksg_tile, dbg_mi, dbg_eps,
                      dbg_nx, dbg_ny,
                      ctx->count_evals ? ctx->evals.as<unsigned long long>() : nullptr, variant,
                      dbg_ey);
}

static ndf_status mi_ksg_variant(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx,
                                 int k, float* out, int variant) {
    if (!ctx) return NDF_ERR_ARG;
    const Field *rf, *qf;
    ndf_status st = check_pair(ctx, ref_field, query_field, ref_idx, &rf, &qf);
    if (st != NDF_OK) return st;
    if ((st = check_ksg_args(ctx, rf, k)) != NDF_OK) return st;
    cudaSetDevice(ctx->device);
    if ((st = ensure_psi_table(ctx, rf->M + 1)) != NDF_OK) return st;
    cudaError_t es = ensure_sorted_columns(ctx, ctx->fields[query_field]);
    if (es != cudaSuccess) return cuda_fail(ctx, es, "sorted columns");
    size_t bytes = sizeof(float) * (size_t)qf->N;
    void* dev_out;
    bool is_host;
    if ((st = resolve_out(ctx, out, bytes, &dev_out, &is_host)) != NDF_OK) return st;
    cudaError_t e = run_ksg_one(ctx, *rf, *qf, ref_idx, k, 0, qf->N, (float*)dev_out, nullptr,
                                nullptr, nullptr, nullptr, variant);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ksg launch");
    return finish_out(ctx, out, dev_out, bytes, is_host);
}

ndf_status ndf_mi_ksg(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx, int k,
                      float* out) {
    return mi_ksg_variant(ctx, ref_field, query_field, ref_idx, k, out, 1);
}

ndf_status ndf_mi_ksg2(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx, int k,
                       float* out) {
    return mi_ksg_variant(ctx, ref_field, query_field, ref_idx, k, out, 2);
}

static ndf_status ksg_debug_variant(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx,
                                    int64_t query_idx, int k, float* eps, float* ey, int32_t* nx,
                                    int32_t* ny, double* mi, int variant) {
    if (!ctx) return NDF_ERR_ARG;
    const Field *rf, *qf;
    ndf_status st = check_pair(ctx, ref_field, query_field, ref_idx, &rf, &qf);
    if (st != NDF_OK) return st;
    if (query_idx < 0 || query_idx >= qf->N) return fail(ctx, NDF_ERR_ARG, "query_idx out of range");
    if ((st = check_ksg_args(ctx, rf, k)) != NDF_OK) return st;
    cudaSetDevice(ctx->device);
    if ((st = ensure_psi_table(ctx, rf->M + 1)) != NDF_OK) return st;
    cudaError_t es = ensure_sorted_columns(ctx, ctx->fields[query_field]);
    if (es != cudaSuccess) return cuda_fail(ctx, es, "sorted columns");
    int64_t M = rf->M;
    // layout of the debug block: mi (double) | out (float) | eps[M] | nx[M] | ny[M] | ey[M]
    size_t need = 16 + sizeof(float) * (size_t)M * 4 + 64;
    cudaError_t e = ctx->dbg.reserve(need);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "debug buffer");
    char* base = ctx->dbg.as<char>();
    double* d_mi = (double*)base;
    float* d_out = (float*)(base + 8);
    float* d_eps = (float*)(base + 16);
    int32_t* d_nx = (int32_t*)(d_eps + M);
    int32_t* d_ny = d_nx + M;
    float* d_ey = (float*)(d_ny + M);
    e = run_ksg_one(ctx, *rf, *qf, ref_idx, k, query_idx, query_idx + 1, d_out, d_mi, d_eps, d_nx,
                    d_ny, variant, d_ey);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ksg debug launch");
    std::vector<char> h(need);
    e = cudaMemcpyAsync(h.data(), base, need, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ksg debug copy");
    const char* hb = h.data();
    if (mi) memcpy(mi, hb, sizeof(double));
    if (eps) memcpy(eps, hb + 16, sizeof(float) * (size_t)M);
    if (nx) memcpy(nx, hb + 16 + 4 * M, sizeof(int32_t) * (size_t)M);
    if (ny) memcpy(ny, hb + 16 + 8 * M, sizeof(int32_t) * (size_t)M);
    if (ey) memcpy(ey, hb + 16 + 12 * M, sizeof(float) * (size_t)M);
    return NDF_OK;
}

ndf_status ndf_ksg_debug_pair(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx,
                              int64_t query_idx, int k, float* eps, int32_t* nx, int32_t* ny,
                              double* mi) {
    return ksg_debug_variant(ctx, ref_field, query_field, ref_idx, query_idx, k, eps, nullptr, nx,
                             ny, mi, 1);
}

ndf_status ndf_ksg2_debug_pair(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx,
                               int64_t query_idx, int k, float* ex, float* ey, int32_t* nx,
                               int32_t* ny, double* mi) {
    return ksg_debug_variant(ctx, ref_field, query_field, ref_idx, query_idx, k, ex, ey, nx, ny,
                             mi, 2);
}

ndf_status ndf_set_ksg_algorithm(ndf_ctx* ctx, int algorithm, int count_evals) {
    if (!ctx) return NDF_ERR_ARG;
    if (algorithm != NDF_KSG_BRUTE && algorithm != NDF_KSG_PRUNED && algorithm != NDF_KSG_BLOCK &&
        algorithm != NDF_KSG_LANES)
        return fail(ctx, NDF_ERR_ARG, "unknown KSG algorithm %d", algorithm);
    ctx->ksg_algorithm = algorithm;
    ctx->count_evals = count_evals != 0;
    if (ctx->count_evals) {
        cudaError_t e = ctx->evals.reserve(sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->evals.ptr, 0, sizeof(unsigned long long), ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "evaluation counter");
    }
    return NDF_OK;
}

ndf_status ndf_ksg_set_schedule(ndf_ctx* ctx, int switch_min, int every) {
    if (!ctx) return NDF_ERR_ARG;
    if (switch_min < 1 || switch_min > 32)
        return fail(ctx, NDF_ERR_ARG, "switch_min %d outside 1..32", switch_min);
    if (every < 1 || every > 8) return fail(ctx, NDF_ERR_ARG, "every %d outside 1..8", every);
    ctx->ksg_switch_min = switch_min;
    ctx->ksg_every = every;
    return NDF_OK;
}

ndf_status ndf_ksg_take_eval_count(ndf_ctx* ctx, uint64_t* out) {
    if (!ctx || !out) return NDF_ERR_ARG;
    *out = 0;
    if (!ctx->count_evals || !ctx->evals.ptr) return NDF_OK;
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, ctx->evals.ptr, sizeof v, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->evals.ptr, 0, sizeof v, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "evaluation counter read");
    *out = v;
    return NDF_OK;
}

ndf_status ndf_mi_ksg_batch(ndf_ctx* ctx, int ref_field, int query_field, const int64_t* ref_idx,
                            int R, int k, float* out) {
    if (!ctx) return NDF_ERR_ARG;
    if (!ref_idx || R < 1) return fail(ctx, NDF_ERR_ARG, "need R >= 1 reference indices");
    const Field *rf, *qf;
    ndf_status st = check_pair(ctx, ref_field, query_field, 0, &rf, &qf);
    if (st != NDF_OK) return st;
    const bool dev_refs = pointer_kind(ref_idx) == PTR_DEVICE;  // checked by the stage kernel
    if (!dev_refs)
        for (int i = 0; i < R; ++i)
            if (ref_idx[i] < 0 || ref_idx[i] >= rf->N)
                return fail(ctx, NDF_ERR_ARG, "ref_idx[%d] out of range", i);
    if ((st = check_ksg_args(ctx, rf, k)) != NDF_OK) return st;
    cudaSetDevice(ctx->device);
    if ((st = ensure_psi_table(ctx, rf->M + 1)) != NDF_OK) return st;
    cudaError_t es = ensure_sorted_columns(ctx, ctx->fields[query_field]);
    if (es != cudaSuccess) return cuda_fail(ctx, es, "sorted columns");
    const size_t bytes = sizeof(float) * (size_t)R * (size_t)qf->N;
    void* dev_out;
    bool is_host;
    if ((st = resolve_out(ctx, out, bytes, &dev_out, &is_host)) != NDF_OK) return st;
    cudaError_t e = cudaSuccess;
    const int64_t* d_refs = ref_idx;
    if (!dev_refs) {
        e = ctx->refidx.reserve(sizeof(int64_t) * (size_t)R);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->refidx.ptr, ref_idx, sizeof(int64_t) * (size_t)R,
                                cudaMemcpyHostToDevice, ctx->stream);
        d_refs = ctx->refidx.as<int64_t>();
    }
    if (e == cudaSuccess)
        e = launch_ksg(ctx, *rf, *qf, d_refs, 0, R, k, 0, qf->N,
                       static_cast<float*>(dev_out), qf->N, ctx->ksg_algorithm != NDF_KSG_BRUTE,
                       ctx->ksg_group, ctx->ksg_tile, nullptr, nullptr, nullptr, nullptr,
                       ctx->count_evals ? ctx->evals.as<unsigned long long>() : nullptr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ksg batch launch");
    return finish_out(ctx, out, dev_out, bytes, is_host);
}

}  // extern "C"
