// Statistical equilibrium of a multi-level molecule (Sec. 2.1.3, Eq.
// boltzmann generalised to n levels) and the pieces of the Lambda iteration
// that run per cell: one thread per cell, FP64.
//
// Rates for each pair u > l: collisions C_ul = k_ul n_coll and, by detailed
// balance, C_lu = (g_u/g_l) C_ul exp(-(E_u - E_l)/T); radiation l -> u at the
// Monte Carlo absorption rate Gamma_lu, u -> l at A_ul + (g_l/g_u) Gamma_lu
// (spontaneous plus stimulated emission). The steady state sum_j n_j R_ji =
// n_i sum_j R_ij, with the last equation replaced by sum_i n_i = n_mol, is
// solved by Gaussian elimination with partial pivoting.
#include <math.h>

#include "krl_internal.cuh"

namespace krl {

namespace {

__global__ void k_lte(LevelConst L, const float* n_mol, int ncell, double* pops)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    double w[kMaxLevels], z = 0.0;
    for (int i = 0; i < L.n; ++i) {
        w[i] = L.g[i] * exp(-(L.E[i] - L.E[0]) / L.T);
        z += w[i];
    }
    const double nm = (double)n_mol[c];
    for (int i = 0; i < L.n; ++i) pops[(size_t)c * L.n + i] = nm * w[i] / z;
}

__global__ void k_level_field(const double* pops, int ncell, int n_lev, int lev, double scale, float* out)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    out[c] = (float)(scale * pops[(size_t)c * n_lev + lev]);
}

// FP64 sum of n_u A over cells into *total, in a fixed order (so the result
// does not depend on scheduling): kSumBlocks blocks each sum a grid-strided
// share into partials[block], then one block sums the partials.
constexpr int kSumBlocks = 512;

__device__ __forceinline__ double block_sum256(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    return sh[0];
}

__global__ void k_sum_rate_part(const double* pops, int ncell, int n_lev, int u, double A, double* partials)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x)
        s += pops[(size_t)c * n_lev + u] * A;
    const double b = block_sum256(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

__global__ void k_sum_rate_final(const double* partials, int n, double* total)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    const double b = block_sum256(s, sh);
    if (threadIdx.x == 0) *total = b;
}

// Gamma_c = (L / N) sigma0 exc_c / dx^2 with L = total * dx^3 photons/s.
__global__ void k_gamma(const double* exc, int ncell, const double* total, double dx, double sigma0, double n_packets,
                        double* gamma)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double Lum = (*total) * dx * dx * dx;
    gamma[c] = Lum / n_packets * sigma0 * exc[c] / (dx * dx);
}

__global__ void k_solve(LevelConst L, const double* gamma, int ncell, const float* n_coll, const float* n_mol,
                        double* pops, unsigned long long* max_change)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int n = L.n;
    double R[kMaxLevels][kMaxLevels];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) R[i][j] = 0.0;
    const double nc = n_coll ? (double)n_coll[c] : 0.0;
    for (int u = 1; u < n; ++u)
        for (int l = 0; l < u; ++l) {
            const double Cul = L.k[u][l] * nc;
            const double Clu = L.g[u] / L.g[l] * Cul * exp(-(L.E[u] - L.E[l]) / L.T);
            R[u][l] += L.A[u][l] + Cul;
            R[l][u] += Clu;
        }
    for (int t = 0; t < L.n_trans; ++t) {
        const int u = L.tu[t], l = L.tl[t];
        const double G = gamma[(size_t)t * ncell + c];
        R[l][u] += G;
        R[u][l] += L.g[l] / L.g[u] * G;
    }
    // M[i][j] = R[j][i] (i != j), M[i][i] = -sum_j R[i][j]; last row: conservation
    double M[kMaxLevels][kMaxLevels + 1];
    for (int i = 0; i < n; ++i) {
        double out = 0.0;
        for (int j = 0; j < n; ++j) {
            M[i][j] = (i == j) ? 0.0 : R[j][i];
            if (j != i) out += R[i][j];
        }
        M[i][i] = -out;
        M[i][n] = 0.0;
    }
    const double nm = (double)n_mol[c];
    for (int j = 0; j < n; ++j) M[n - 1][j] = 1.0;
    M[n - 1][n] = nm;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double best = fabs(M[col][col]);
        for (int r = col + 1; r < n; ++r)
            if (fabs(M[r][col]) > best) { best = fabs(M[r][col]); piv = r; }
        if (piv != col)
            for (int j = 0; j <= n; ++j) { double t = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = t; }
        const double d = M[col][col];
        if (d == 0.0) continue;             // singular (n_mol = 0 cell): leaves zeros
        for (int r = col + 1; r < n; ++r) {
            const double f = M[r][col] / d;
            if (f != 0.0)
                for (int j = col; j <= n; ++j) M[r][j] -= f * M[col][j];
        }
    }
    double x[kMaxLevels];
    for (int i = n - 1; i >= 0; --i) {
        double s = M[i][n];
        for (int j = i + 1; j < n; ++j) s -= M[i][j] * x[j];
        x[i] = M[i][i] != 0.0 ? s / M[i][i] : 0.0;
    }
    double change = 0.0;
    for (int i = 0; i < n; ++i) {
        double* p = pops + (size_t)c * n + i;
        const double old = *p;
        const double v = x[i] > 0.0 ? x[i] : 0.0;     // round-off below zero
        if (nm > 0.0) change = fmax(change, fabs(v - old) / nm);
        *p = v;
    }
    if (max_change) atomicMax(max_change, (unsigned long long)__double_as_longlong(change));
}

}  // namespace

cudaError_t levels_lte(const LevelConst& L, const float* n_mol, int ncell, double* pops, cudaStream_t s)
{
    k_lte<<<(ncell + 255) / 256, 256, 0, s>>>(L, n_mol, ncell, pops);
    return cudaGetLastError();
}

cudaError_t levels_field(const double* pops, int ncell, int n_lev, int lev, double scale, float* out, cudaStream_t s)
{
    k_level_field<<<(ncell + 255) / 256, 256, 0, s>>>(pops, ncell, n_lev, lev, scale, out);
    return cudaGetLastError();
}

size_t levels_sum_scratch_doubles() { return 1 + (size_t)kSumBlocks; }

cudaError_t levels_sum_rate(const double* pops, int ncell, int n_lev, int u, double A, double* total, cudaStream_t s)
{
    k_sum_rate_part<<<kSumBlocks, 256, 0, s>>>(pops, ncell, n_lev, u, A, total + 1);
    k_sum_rate_final<<<1, 256, 0, s>>>(total + 1, kSumBlocks, total);
    return cudaGetLastError();
}

cudaError_t levels_gamma(const double* exc, int ncell, const double* total, double dx, double sigma0, double n_packets,
                         double* gamma, cudaStream_t s)
{
    k_gamma<<<(ncell + 255) / 256, 256, 0, s>>>(exc, ncell, total, dx, sigma0, n_packets, gamma);
    return cudaGetLastError();
}

cudaError_t levels_solve(const LevelConst& L, const double* gamma, int ncell, const float* n_coll, const float* n_mol,
                         double* pops, unsigned long long* max_change, cudaStream_t s)
{
    k_solve<<<(ncell + 127) / 128, 128, 0, s>>>(L, gamma, ncell, n_coll, n_mol, pops, max_change);
    return cudaGetLastError();
}

}  // namespace krl
