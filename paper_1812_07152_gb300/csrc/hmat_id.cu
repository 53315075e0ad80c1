// Nested row interpolative decompositions on the GPU (the low-rank approximation of
// Section 3.1, batched): one CTA per tree node of a level. Each CTA forms A = K(C, R)
// (|C| sampled far points x |R| candidate rows, column-major, FP64) from the points,
// runs a column-pivoted Householder QR of it, stopped at the first pivot |R_kk| <=
// tol |R_11| or at the rank cap, and solves T = R_11^{-1} R_12 in place. The host turns
// (pivots, T) into the skeleton and the basis P = Pi [I; T^T]. The steps are those of
// the host inspector's row ID (first maximum pivot, LAPACK-style reflectors and norm
// downdating with recomputation on cancellation); only the order of the sums differs.
#include <cuda_runtime.h>

#include <vector>

#include "hmat_internal.h"

namespace hmat {
namespace {

constexpr int kIdThreads = 256;
constexpr int kIdWarps = kIdThreads / 32;

__device__ double kernel_value_d(int kernel, double param, const double* x, const double* y, int d) {
  double r2 = 0.0;
  for (int k = 0; k < d; ++k) {
    const double diff = __dsub_rn(x[k], y[k]);
    r2 = __dadd_rn(r2, __dmul_rn(diff, diff));
  }
  if (kernel == HMAT_KERNEL_GAUSSIAN) return exp(-r2 / (2.0 * param * param));
  if (kernel == HMAT_KERNEL_IMQ) return 1.0 / sqrt(r2 + param * param);
  return r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA; every thread gets the result.
__device__ double cta_sum(double v, double* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kIdWarps; ++w) s += red[w];
  return s;
}

__global__ void __launch_bounds__(kIdThreads) k_row_id(const IdJob* __restrict__ jobs, const double* __restrict__ pts,
                                                       int d, const int64_t* __restrict__ ids, int kernel,
                                                       double param, double tol, int max_rank,
                                                       double* __restrict__ work, int32_t* __restrict__ piv_out,
                                                       int32_t* __restrict__ rank_out) {
  extern __shared__ double sm[];
  __shared__ double red[kIdWarps];
  __shared__ int red_i[kIdWarps];
  __shared__ double red_v[kIdWarps];
  const IdJob job = jobs[blockIdx.x];
  const int64_t n = job.n_rows, m = job.n_cols;
  double* A = work + job.a_off;
  int32_t* piv = piv_out + job.piv_off;
  double* vn1 = sm;
  double* vn2 = sm + n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (n == 0 || m == 0) {
    if (tid == 0) rank_out[blockIdx.x] = 0;
    return;
  }
  if (pts) {  // else A is given (hmat_selftest_row_id)
    const int64_t* rows = ids + job.rows_off;
    const int64_t* cols = ids + job.cols_off;
    // A[j * m + i] = k(x_{cols[i]}, x_{rows[j]})
    for (int64_t e = tid; e < n * m; e += kIdThreads) {
      const int64_t j = e / m, i = e % m;
      A[e] = kernel_value_d(kernel, param, pts + cols[i] * d, pts + rows[j] * d, d);
    }
  }
  for (int64_t j = tid; j < n; j += kIdThreads) piv[j] = (int32_t)j;
  __syncthreads();
  for (int64_t j = warp; j < n; j += kIdWarps) {
    double s = 0.0;
    for (int64_t i = lane; i < m; i += 32) s += A[j * m + i] * A[j * m + i];
    s = warp_sum(s);
    if (lane == 0) vn1[j] = vn2[j] = sqrt(s);
  }
  __syncthreads();
  const double tol3z = sqrt(2.220446049250313e-16);
  const int64_t kmax = min((int64_t)max_rank, min(n, m));
  double r11 = 0.0;
  int64_t k = 0;
  for (; k < kmax; ++k) {
    // pivot: the first largest partial norm among columns k..n-1
    double bv = -1.0;
    int bi = (int)n;
    for (int64_t j = k + tid; j < n; j += kIdThreads)
      if (vn1[j] > bv) { bv = vn1[j]; bi = (int)j; }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    __syncthreads();
    if (lane == 0) { red_v[warp] = bv; red_i[warp] = bi; }
    __syncthreads();
    int p = (int)n;
    double pv = -1.0;
    for (int w = 0; w < kIdWarps; ++w)
      if (red_v[w] > pv || (red_v[w] == pv && red_i[w] < p)) { pv = red_v[w]; p = red_i[w]; }
    if (p != k && p < n) {
      for (int64_t i = tid; i < m; i += kIdThreads) {
        const double t = A[p * m + i];
        A[p * m + i] = A[k * m + i];
        A[k * m + i] = t;
      }
      __syncthreads();
      if (tid == 0) {
        const int32_t t = piv[p];
        piv[p] = piv[k];
        piv[k] = t;
        vn1[p] = vn1[k];
        vn2[p] = vn2[k];
      }
    }
    __syncthreads();
    // Householder reflector of A[k:m, k]
    double* col = A + k * m;
    const double alpha = col[k];
    double xs = 0.0;
    for (int64_t i = k + 1 + tid; i < m; i += kIdThreads) xs += col[i] * col[i];
    const double xn = sqrt(cta_sum(xs, red));
    double beta = alpha, tau = 0.0;
    if (xn != 0.0) {
      beta = -copysign(hypot(alpha, xn), alpha);
      tau = (beta - alpha) / beta;
      const double scal = 1.0 / (alpha - beta);
      for (int64_t i = k + 1 + tid; i < m; i += kIdThreads) col[i] *= scal;
    }
    __syncthreads();
    if (tid == 0) col[k] = beta;
    const double rkk = fabs(beta);
    if (k == 0) r11 = rkk;
    if (!(rkk > tol * r11) || r11 == 0.0) break;  // CTA-uniform: every thread saw the same beta
    __syncthreads();
    // apply (I - tau v v^T), v = [1; col[k+1:m]], to the columns k+1..n-1 (one warp per column)
    if (tau != 0.0)
      for (int64_t j = k + 1 + warp; j < n; j += kIdWarps) {
        double* cj = A + j * m;
        double w = 0.0;
        for (int64_t i = k + 1 + lane; i < m; i += 32) w += col[i] * cj[i];
        w = (warp_sum(w) + cj[k]) * tau;
        if (lane == 0) cj[k] -= w;
        for (int64_t i = k + 1 + lane; i < m; i += 32) cj[i] -= w * col[i];
      }
    __syncthreads();
    // downdate the partial column norms (recompute on large cancellation)
    for (int64_t j = k + 1 + warp; j < n; j += kIdWarps) {
      if (vn1[j] == 0.0) continue;
      const double r = fabs(A[j * m + k]) / vn1[j];
      const double temp = fmax(0.0, (1.0 + r) * (1.0 - r));
      const double ratio = vn1[j] / vn2[j];
      if (temp * ratio * ratio <= tol3z) {
        double s = 0.0;
        for (int64_t i = k + 1 + lane; i < m; i += 32) s += A[j * m + i] * A[j * m + i];
        s = warp_sum(s);
        __syncwarp();
        if (lane == 0) vn1[j] = vn2[j] = sqrt(s);
      } else if (lane == 0) {
        vn1[j] *= sqrt(temp);
      }
      __syncwarp();
    }
    __syncthreads();
  }
  __syncthreads();
  // T = R_11^{-1} R_12 in place of R_12: column c of T overwrites rows 0..k-1 of column k+c
  for (int64_t c = tid; c < n - k; c += kIdThreads) {
    double* tc = A + (k + c) * m;
    for (int64_t i = k - 1; i >= 0; --i) {
      double s = tc[i];
      for (int64_t j = i + 1; j < k; ++j) s -= A[j * m + i] * tc[j];
      tc[i] = s / A[i * m + i];
    }
  }
  if (tid == 0) rank_out[blockIdx.x] = (int32_t)k;
}

}  // namespace

cudaError_t launch_row_id(const IdJob* jobs, int64_t n_jobs, int64_t max_rows, const double* pts, int d,
                          const int64_t* ids, int kernel, double param, double tol, int max_rank, double* work,
                          int32_t* piv, int32_t* rank, cudaStream_t stream) {
  if (n_jobs == 0) return cudaSuccess;
  if (n_jobs > 2147483647LL) return cudaErrorInvalidValue;
  const size_t smem = (size_t)(2 * max_rows) * sizeof(double);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_row_id, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_row_id<<<(unsigned)n_jobs, kIdThreads, smem, stream>>>(jobs, pts, d, ids, kernel, param, tol, max_rank, work,
                                                            piv, rank);
  return cudaGetLastError();
}

}  // namespace hmat

using namespace hmat;

extern "C" hmat_status hmat_selftest_row_id(const double* M, int64_t n_rows, int64_t n_cols, double tol,
                                            int32_t max_rank, int32_t* piv, int32_t* rank, double* T) {
  if (!M || !piv || !rank || !T || n_rows <= 0 || n_cols <= 0 || max_rank < 1 || !(tol >= 0.0)) return HMAT_EINVAL;
  if (n_rows > 8192 || n_rows * n_cols > ((int64_t)1 << 26)) return HMAT_EINVAL;
  const int64_t vals = n_rows * n_cols;
  double* dA = nullptr;
  int32_t* dp = nullptr;
  int32_t* dr = nullptr;
  IdJob* dj = nullptr;
  const IdJob job{0, 0, 0, 0, (int32_t)n_rows, (int32_t)n_cols};
  cudaError_t e = cudaMalloc((void**)&dA, (size_t)vals * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dp, (size_t)n_rows * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dr, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dj, sizeof(IdJob));
  // column j of the column-major |C| x |R| operand is row j of M
  if (e == cudaSuccess) e = cudaMemcpy(dA, M, (size_t)vals * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dj, &job, sizeof(IdJob), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = launch_row_id(dj, 1, n_rows, nullptr, 0, nullptr, 0, 0.0, tol, max_rank, dA, dp, dr, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int32_t k = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&k, dr, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(piv, dp, (size_t)n_rows * sizeof(int32_t), cudaMemcpyDeviceToHost);
  std::vector<double> A;
  if (e == cudaSuccess) {
    A.resize((size_t)vals);
    e = cudaMemcpy(A.data(), dA, (size_t)vals * sizeof(double), cudaMemcpyDeviceToHost);
  }
  cudaFree(dA);
  cudaFree(dp);
  cudaFree(dr);
  cudaFree(dj);
  if (e != cudaSuccess) return cuda_status(e);
  *rank = k;
  // T (k x (n_rows - k), row-major): column c sits in rows 0..k-1 of column k + c
  for (int64_t i = 0; i < k; ++i)
    for (int64_t c = 0; c < n_rows - k; ++c) T[i * (n_rows - k) + c] = A[(size_t)((k + c) * n_cols + i)];
  return HMAT_OK;
}
