// Internal declarations shared by the CUDA translation units of libndf.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ndf.h"

namespace ndf {

// A device allocation owned by the context; grows on demand, never shrinks.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t need);
    void release();
    template <class T>
    T* as() const { return static_cast<T*>(ptr); }
};

struct Field {
    bool live = false;
    int64_t M = 0, Z = 0, Y = 0, X = 0, N = 0;
    float* data = nullptr;     // [M][N]
    double* mean = nullptr;    // [N]
    double* inv_norm = nullptr;// [N] 1/sqrt(sum (e - mean)^2), 0 when the sum is 0
    // standardised vertex-major copies for the tensor-core batched Pearson
    // (built on first use): z[v][m] = (e_m(v) - mean_v) * inv_norm_v, m < Kp
    int Kp = 0;
    void* z_tf32 = nullptr;    // float [N][Kp], TF32-rounded
    void* z_hi = nullptr;      // bf16 [N][Kp]
    void* z_lo = nullptr;      // bf16 [N][Kp]
    // every vertex column sorted ascending, member-major like `data` (built on
    // the first KSG call that uses this field as the query field)
    float* sorted = nullptr;   // [M][N]
    void free_all();
};

}  // namespace ndf

struct ndf_ctx {
    struct CachedBuf {
        void* ptr;
        size_t bytes;
    };
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    cudaStream_t copy_stream = nullptr;  // uploads, overlapped with per-chunk statistics
    cudaEvent_t copy_event = nullptr;
    std::vector<ndf::Field> fields;
    std::string last_error;
    uint64_t launches = 0;
    // scratch
    ndf::DevBuf stage_x;     // reference column: centred values (Pearson) / sorted values (KSG)
    ndf::DevBuf stage_perm;  // KSG: member index of each sorted position
    ndf::DevBuf out_tmp;     // device output staging when the caller passes host memory
    ndf::DevBuf psi;         // digamma table psi(0..psi_n-1), FP64
    int64_t psi_n = 0;
    ndf::DevBuf dbg;         // KSG debug outputs
    ndf::DevBuf flag;        // small device status words
    int ksg_algorithm = NDF_KSG_LANES;
    int ksg_group = 4;       // references per CTA in batched KSG (tuned by ndf_ksg_autotune)
    int ksg_tile = 8;        // query vertices per tile
    int ksg_switch_min = 12; // lane-refill search: waiting lanes that start a service step
    int ksg_every = 5;       // lane-refill search: scan steps between service checks
    bool count_evals = false;
    ndf::DevBuf evals;       // KSG distance evaluations (when counting is on)
    ndf::DevBuf ksg_work;    // pruned KSG: work-item counter
    ndf::DevBuf render_buf;  // ray-march: transfer function and uploaded host volumes
    std::vector<CachedBuf> cache;  // device buffers of freed fields, reused by later loads
    ndf::DevBuf zr;          // batched Pearson: standardised reference rows
    ndf::DevBuf refidx;      // batched calls: reference indices on the device
    ndf::DevBuf col_data;    // volumes against an external reference column: the column
    ndf::DevBuf col_stats;   //   its mean, 1/sqrt(S) and a non-finite flag
    ndf::Field col_field;    //   the one-vertex reference field over those buffers
};

namespace ndf {

enum PtrKind { PTR_HOST = 0, PTR_DEVICE = 1 };

// Field buffers go through the context's cache: ctx_alloc takes a cached buffer of
// exactly `bytes` if there is one (else cudaMalloc, trimming the cache and retrying
// on out-of-memory); ctx_release keeps the buffer (at most kCacheEntries, the
// oldest freed beyond that); ctx_trim frees every cached buffer.
constexpr size_t kCacheEntries = 8;
cudaError_t ctx_alloc(ndf_ctx* ctx, void** p, size_t bytes);
void ctx_release(ndf_ctx* ctx, void* p, size_t bytes);
void ctx_trim(ndf_ctx* ctx);
// Returns a field's buffers to the cache (standardised copies are freed) and marks it dead.
void release_field(ndf_ctx* ctx, Field& f);
PtrKind pointer_kind(const void* p);

ndf_status fail(ndf_ctx* ctx, ndf_status st, const char* fmt, ...);
ndf_status cuda_fail(ndf_ctx* ctx, cudaError_t e, const char* what);

// Validates field ids, shapes and the reference index; on success returns the fields.
ndf_status check_pair(ndf_ctx* ctx, int ref_field, int query_field, int64_t ref_idx,
                      const Field** rf, const Field** qf);

// Resolves an output pointer: device pointers are used directly, host pointers
// get a context-owned device staging buffer of `bytes`.
ndf_status resolve_out(ndf_ctx* ctx, void* out, size_t bytes, void** dev_out, bool* is_host);
ndf_status check_device_status(ndf_ctx* ctx);
ndf_status finish_out(ndf_ctx* ctx, void* out, const void* dev_out, size_t bytes, bool is_host);

// Digamma psi(n) for n = 0..n_max (entry 0 unused), FP64, on the device.
ndf_status ensure_psi_table(ndf_ctx* ctx, int64_t n_max);
double digamma_int_host(int64_t n);

// kernels (launch wrappers; each returns the launch error)
// (on `stream`, the context's stream when null)
cudaError_t launch_field_stats(ndf_ctx* ctx, const Field& f, int64_t v_begin, int64_t v_end,
                               int* d_nonfinite, cudaStream_t stream = nullptr);
cudaError_t launch_pearson(ndf_ctx* ctx, const Field& rf, const Field& qf, int64_t ref_idx,
                           float* out);
// KSG MI for R references (d_refs on the device, or references ref0, ref0 + 1, ...
// when d_refs is null) against query vertices [v_begin, v_end):
// out[r * out_stride + (v - v_begin)].  prune selects the exact pruned scan over
// brute force; G references share a CTA's query tile of VT vertices.  paired:
// only the pairs (reference i, vertex v_begin + i), out[i], R = v_end - v_begin.
cudaError_t launch_ksg(ndf_ctx* ctx, const Field& rf, const Field& qf, const int64_t* d_refs,
                       int64_t ref0, int R, int k, int64_t v_begin, int64_t v_end, float* out,
                       int64_t out_stride, bool prune, int G, int VT, double* dbg_mi,
                       float* dbg_eps, int32_t* dbg_nx, int32_t* dbg_ny,
                       unsigned long long* evals, int variant = 1, float* dbg_ey = nullptr,
                       bool paired = false);

// Builds Field::sorted (one sort per vertex column, kept with the field).
cudaError_t ensure_sorted_columns(ndf_ctx* ctx, Field& f);
// Sorts the columns of vertices [v_begin, v_end) into the allocated Field::sorted.
// Up to kSortTileMaxM members the kernel can do two more things on the way:
//  - with src (a device field of f's shape) the columns are read from src and also
//    written unsorted into f.data: the copy of a device-resident field;
//  - with d_nonfinite it writes the statistics of launch_field_stats (f.mean,
//    f.inv_norm, the flag set on a non-finite member) from the same registers.
// Either above kSortTileMaxM: cudaErrorInvalidValue.
constexpr int kSortTileMaxM = 1024;
struct ColumnStats {
    double* mean;
    double* inv_norm;
    int* nonfinite;
};
cudaError_t launch_sort_columns(ndf_ctx* ctx, const Field& f, int64_t v_begin, int64_t v_end,
                                cudaStream_t stream, const float* src = nullptr,
                                int* d_nonfinite = nullptr);

// Scratch of the continuous sampler: position, column and statistics blocks for
// up to `cap` pairs, reused across calls.
struct SampleScratch {
    float *ca = nullptr, *cb = nullptr, *cb_sorted = nullptr;
    double *ma = nullptr, *sa = nullptr, *mb = nullptr, *sb = nullptr;
    int64_t cap = 0, M = 0;
    void release() {
        void* ps[] = {ca, cb, cb_sorted, ma, sa, mb, sb};
        for (void* q : ps)
            if (q) cudaFree(q);
        *this = SampleScratch();
    }
    cudaError_t reserve(int64_t M_, int64_t n) {
        if (n <= cap && M_ == M) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&ca, sizeof(float) * (size_t)M_ * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&cb, sizeof(float) * (size_t)M_ * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&cb_sorted, sizeof(float) * (size_t)M_ * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&ma, sizeof(double) * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&sa, sizeof(double) * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&mb, sizeof(double) * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&sb, sizeof(double) * (size_t)n);
        if (e != cudaSuccess) {
            release();
            return e;
        }
        cap = n;
        M = M_;
        return cudaSuccess;
    }
};

// n continuous-position training triples (Sec. 4.3) into device arrays
// pref[n][3], pq[n][3], target[n] (ndf_sample_triples without the host side).
cudaError_t sample_triples_dev(ndf_ctx* ctx, const Field& rf, const Field& qf, int measure, int k,
                               int64_t n, uint64_t seed, float* pref, float* pq, float* target,
                               SampleScratch& sc);

constexpr int kKsgMaxM = 4096;
constexpr int kKsgMaxK = 16;

}  // namespace ndf
