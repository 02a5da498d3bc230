// dog_eval.cuh -- evaluation of the filter's cell estimates against ground truth (the
// experiments of Sect. VIII): velocity statistics of the cells of an object and the
// Mahalanobis-distance classification of cells into static and dynamic.
#pragma once
#include "dog_common.cuh"

namespace dog {

constexpr int EVAL_BLOCK = 256;

// Per-object sums over the cells of each object (Eq. mean_cluster, gaussian_mixture_x):
// |S|, sum mean_x, sum mean_y, sum (var_x + mean_x^2), sum (var_y + mean_y^2).  Each cell
// term is formed in binary64 (exact products of the binary32 estimates) and added in signed
// 2^-32 fixed point with integer atomics, so the sums do not depend on the order.
__global__ void __launch_bounds__(EVAL_BLOCK) k_eval_cluster_sums(KParams P, DevBufs B, const int32_t *__restrict__ obj,
                                                                  uint32_t n_obj, long long *__restrict__ sums) {
  for (uint32_t c = blockIdx.x * EVAL_BLOCK + threadIdx.x; c < P.C; c += gridDim.x * EVAL_BLOCK) {
    const int32_t k = __ldg(obj + c);
    if (k <= 0 || (uint32_t)k > n_obj) continue;
    const double mx = B.mean_x[c], my = B.mean_y[c];
    const double tx = (double)B.var_x[c] + mx * mx, ty = (double)B.var_y[c] + my * my;
    long long *s = sums + (size_t)(k - 1) * 5;
    atomicAdd(reinterpret_cast<unsigned long long *>(s), 1ull);
    const double v[4] = {mx, my, tx, ty};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      atomicAdd(reinterpret_cast<unsigned long long *>(s + 1 + j),
                (unsigned long long)__double2ll_rz(v[j] * 4294967296.0));
  }
}

// statistics of each object from its sums: |S|, mean vx, mean vy, var vx, var vy
__global__ void k_eval_cluster_stats(const long long *__restrict__ sums, uint32_t n_obj, double *__restrict__ st) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_obj; k += gridDim.x * blockDim.x) {
    const long long *s = sums + (size_t)k * 5;
    const double n = (double)s[0];
    double *o = st + (size_t)k * 5;
    o[0] = n;
    if (s[0] == 0) {
      o[1] = o[2] = o[3] = o[4] = 0.0;
      continue;
    }
    const double q = 1.0 / 4294967296.0;
    const double mx = (double)s[1] * q / n, my = (double)s[2] * q / n;
    o[1] = mx;
    o[2] = my;
    o[3] = (double)s[3] * q / n - mx * mx;
    o[4] = (double)s[4] * q / n - my * my;
  }
}

// Mahalanobis distance of the cell's Gaussian velocity estimate from v = 0 (Eq. mahadist),
// m = v P^-1 v^T with P = [[var_x, cov], [cov, var_y]], in binary32 with a fixed order:
// (var_y vx^2 - 2 cov vx vy + var_x vy^2) / (var_x var_y - cov^2); a singular P gives 0 for
// v = 0 and +inf otherwise.
__device__ __forceinline__ float mahalanobis0(float vx, float vy, float sx, float sy, float cv) {
  const float a = __fmul_rn(vx, vx), b = __fmul_rn(vy, vy), c = __fmul_rn(vx, vy);
  const float t2 = __fmul_rn(cv, c);
  const float num = __fadd_rn(__fsub_rn(__fmul_rn(sy, a), __fadd_rn(t2, t2)), __fmul_rn(sx, b));
  const float det = __fsub_rn(__fmul_rn(sx, sy), __fmul_rn(cv, cv));
  if (det > 0.0f) return __fdiv_rn(num, det);
  return (vx == 0.0f && vy == 0.0f) ? 0.0f : __int_as_float(0x7f800000);
}

// Per class (label 1 = dynamic, 2 = static) a histogram of how many of the sorted thresholds
// are <= m over the cells with that label and m_occ >= min_occ; counts[l - 1][j].  m of every
// cell goes to m_out when given (0 for cells not evaluated).
__global__ void __launch_bounds__(EVAL_BLOCK) k_eval_mahalanobis(KParams P, DevBufs B, const uint8_t *__restrict__ label,
                                                                 float min_occ, const float *__restrict__ thr,
                                                                 uint32_t n_thr, unsigned long long *__restrict__ counts,
                                                                 float *__restrict__ m_out) {
  extern __shared__ unsigned int sh_cnt[];  // [2][n_thr + 1]
  const uint32_t nb = n_thr + 1u;
  for (uint32_t k = threadIdx.x; k < 2u * nb; k += EVAL_BLOCK) sh_cnt[k] = 0u;
  __syncthreads();
  for (uint32_t c = blockIdx.x * EVAL_BLOCK + threadIdx.x; c < P.C; c += gridDim.x * EVAL_BLOCK) {
    const uint32_t l = __ldg(label + c);
    float m = 0.0f;
    if ((l == 1u || l == 2u) && B.mO[c] >= min_occ) {
      m = mahalanobis0(B.mean_x[c], B.mean_y[c], B.var_x[c], B.var_y[c], B.cov[c]);
      uint32_t lo = 0, hi = n_thr;  // number of thresholds <= m
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(thr + mid) <= m) lo = mid + 1u; else hi = mid;
      }
      atomicAdd(&sh_cnt[(l - 1u) * nb + lo], 1u);
    }
    if (m_out) m_out[c] = m;
  }
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < 2u * nb; k += EVAL_BLOCK)
    if (sh_cnt[k]) atomicAdd(counts + k, (unsigned long long)sh_cnt[k]);
}

}  // namespace dog
