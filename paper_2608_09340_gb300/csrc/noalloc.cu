// krl_emission_cdf_noalloc: the volume-source emission CDF (the inclusive
// FP64 scan of the per-cell emission rate, normalised by its total, that
// krl_line_set builds for KRL_SRC_VOLUME) computed without allocating any
// device memory.
//
// Some callers cannot call cudaMalloc: a host application that hands all
// device memory to its own pool or framework allocator (so a raw cudaMalloc
// may fail or fragment that pool), or a latency-critical loop that must not
// take cudaMalloc's implicit device synchronisation. For them the scan's
// scratch (per-block partial sums and a validation flag) lives in the
// file-scope array below instead of memory the library allocates. The
// caller still passes the input rates and the output CDF buffer.
#include <stdio.h>

#include <mutex>

#include "krl_internal.cuh"

namespace {

constexpr int kNaMaxCells = 1 << 27;                 // largest grid this entry point accepts
constexpr int kNaT = 256;                            // threads per scan block
constexpr int kNaE = 8;                              // elements per thread
constexpr int kNaChunk = kNaT * kNaE;
constexpr int kNaBlocks = kNaMaxCells / kNaChunk;    // 65536 partial sums
constexpr size_t kNaFlagBytes = 256;                 // validation flag, padded to the alignment
constexpr size_t kNaScratchBytes = kNaFlagBytes + (size_t)(kNaBlocks + 1) * sizeof(double);  // ~512 KiB

// Shared by every call on a device and kept until the process exits; it
// holds the last call's partial sums. Only the flag must start at zero, and
// each call clears it first.
static __device__ __align__(256) unsigned char g_cdf_scratch[kNaScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_cdf_scratch on the current device, looked up once per
// device (the host-side name is only a stand-in, not a device address).
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cdf_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

__device__ double na_block_scan(double v, double* sh)
{
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = 1; off < kNaT; off <<= 1) {
        double add = t >= off ? sh[t - off] : 0.0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    double r = sh[t];
    __syncthreads();
    return r;
}

// Per-block inclusive scans; block totals and the bad-value flag go to scratch.
__global__ void k_na_local(const float* rate, int n, double* out, double* tot, int* bad)
{
    __shared__ double sh[kNaT];
    size_t base = (size_t)blockIdx.x * kNaChunk + (size_t)threadIdx.x * kNaE;
    double v[kNaE];
    double run = 0.0;
    for (int e = 0; e < kNaE; ++e) {
        size_t i = base + e;
        double r = 0.0;
        if (i < (size_t)n) {
            float f = rate[i];
            if (!isfinite(f) || f < 0.0f) atomicOr(bad, 1);
            r = (double)f;
        }
        run += r;
        v[e] = run;
    }
    double incl = na_block_scan(run, sh);
    double excl = incl - run;
    for (int e = 0; e < kNaE; ++e) {
        size_t i = base + e;
        if (i < (size_t)n) out[i] = v[e] + excl;
    }
    if (threadIdx.x == kNaT - 1) tot[blockIdx.x] = incl;
}

// One block: block totals -> exclusive offsets, in place.
__global__ void k_na_offsets(double* tot, int nb)
{
    __shared__ double sh[kNaT];
    int per = (nb + kNaT - 1) / kNaT;
    int b0 = threadIdx.x * per;
    double run = 0.0;
    for (int b = b0; b < b0 + per && b < nb; ++b) run += tot[b];
    double incl = na_block_scan(run, sh);
    double off = incl - run;
    for (int b = b0; b < b0 + per && b < nb; ++b) {
        double t = tot[b];
        tot[b] = off;
        off += t;
    }
}

__global__ void k_na_total(const double* out, int n, double* tot, int nb, int* bad)
{
    double total = out[n - 1] + tot[(n - 1) / kNaChunk];
    tot[nb] = total;
    if (!(total > 0.0)) atomicOr(bad, 2);
}

__global__ void k_na_finish(double* out, int n, const double* tot, int nb)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n) return;
    double total = tot[nb];
    if (!(total > 0.0)) return;
    out[i] = (out[i] + tot[i / kNaChunk]) / total;
}

}  // namespace

namespace krl {
void set_last_error(const char* msg);   // capi.cu: the message krl_last_error() returns
}

namespace {
thread_local char g_na_err[256] = "";
}  // namespace

extern "C" krl_status krl_emission_cdf_noalloc(const float* rate, int n, double* cdf, krl_stream st)
{
    cudaStream_t s = (cudaStream_t)st;
    if (!rate || !cdf) {
        snprintf(g_na_err, sizeof(g_na_err), "krl_emission_cdf_noalloc: NULL rate or cdf");
        return krl::set_last_error(g_na_err), KRL_ERR_ARG;
    }
    if (n < 1 || n > kNaMaxCells) {
        snprintf(g_na_err, sizeof(g_na_err),
                 "krl_emission_cdf_noalloc: n = %d cells is outside [1, %d] (fixed scratch of %zu bytes)", n,
                 kNaMaxCells, kNaScratchBytes);
        return krl::set_last_error(g_na_err), KRL_ERR_ARG;
    }
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        snprintf(g_na_err, sizeof(g_na_err), "krl_emission_cdf_noalloc: scratch address: %s", cudaGetErrorString(e));
        return krl::set_last_error(g_na_err), KRL_ERR_CUDA;
    }
    int* bad = (int*)base;
    double* tot = (double*)((unsigned char*)base + kNaFlagBytes);
    const int nb = (n + kNaChunk - 1) / kNaChunk;
    e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_na_local<<<nb, kNaT, 0, s>>>(rate, n, cdf, tot, bad);
        k_na_offsets<<<1, kNaT, 0, s>>>(tot, nb);
        k_na_total<<<1, 1, 0, s>>>(cdf, n, tot, nb, bad);
        k_na_finish<<<(n + 255) / 256, 256, 0, s>>>(cdf, n, tot, nb);
        e = cudaGetLastError();
    }
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        snprintf(g_na_err, sizeof(g_na_err), "krl_emission_cdf_noalloc: %s", cudaGetErrorString(e));
        return krl::set_last_error(g_na_err), KRL_ERR_CUDA;
    }
    if (hbad & 1) {
        snprintf(g_na_err, sizeof(g_na_err), "krl_emission_cdf_noalloc: rate holds NaN/Inf or a negative value");
        return krl::set_last_error(g_na_err), KRL_ERR_NUMERIC;
    }
    if (hbad & 2) {
        snprintf(g_na_err, sizeof(g_na_err), "krl_emission_cdf_noalloc: rate sums to zero");
        return krl::set_last_error(g_na_err), KRL_ERR_ARG;
    }
    return KRL_OK;
}
