// Static user equilibrium (Waddell et al., Sec. 5.2, Eq. 6) by Frank-Wolfe on BPR link
// times (Eq. 3): the per-link kernels of one iteration.  The direction finding
// (all-or-nothing assignment) is the routing kernel in its counting mode; the host
// side (gbt_api.cu) runs the iteration.
//
// Everything here is binary64 with a fixed operation order per link.  Sums whose value
// steers the iteration (the gap, the sign of the line search's derivative, the
// objective) are exact: each term is rounded to the grid 2^-S (S chosen on the host from
// a bound of the terms so that the total stays below 2^62) and the 64-bit integers are
// added, so neither the atomics' order nor the grid shape can change a decision.
#include "gbt_internal.cuh"

namespace gbt {

#define LS(e, n) for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (n); e += gridDim.x * blockDim.x)

// Eq. 3, t = t0 (1 + alpha (x / c)^beta), beta a small integer (repeated products)
__device__ __forceinline__ double bpr_t(double t0, double x, double c, double alpha, int beta) {
  const double r = x / c;
  double p = 1.0;
  for (int k = 0; k < beta; k++) p = p * r;
  return t0 * (1.0 + alpha * p);
}

// the Beckmann term: integral of Eq. 3 from 0 to x
__device__ __forceinline__ double bpr_area(double t0, double x, double c, double alpha, int beta) {
  const double r = x / c;
  double p = 1.0;
  for (int k = 0; k < beta; k++) p = p * r;
  return t0 * x * (1.0 + alpha * p / (double)(beta + 1));
}

// max of non-negative doubles through their bit patterns (monotone for x >= 0)
__device__ __forceinline__ void max_nonneg(unsigned long long* slot, double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_down_sync(0xffffffffu, b, o);
    b = w > b ? w : b;
  }
  if ((threadIdx.x & 31) == 0 && b) atomicMax(slot, b);
}

// exact integer sum of the warp's terms into slot (two's complement wraps correctly)
__device__ __forceinline__ void add_fixed(unsigned long long* slot, long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(slot, (unsigned long long)v);
}

__global__ void k_fw_t0(const float* len, const float* spd, double* t0, int n) {
  LS(e, n) t0[e] = (double)len[e] / (double)spd[e];   // Eq. 4, seconds
}

__global__ void k_fw_counts(const unsigned* cnt, double* x, int n) {
  LS(e, n) x[e] = (double)cnt[e];
}

__global__ void k_fw_time(const double* t0, const double* x, const double* cap, double alpha, int beta, double* t,
                          unsigned long long* tmax, int n) {
  double m = 0.0;
  LS(e, n) {
    const double v = bpr_t(t0[e], x[e], cap[e], alpha, beta);
    t[e] = v;
    m = v > m ? v : m;
  }
  max_nonneg(tmax, m);
}

__global__ void k_fw_quantize(const double* t, double unit, int qmax, int32_t* q, int n) {
  LS(e, n) {
    double c = floor(t[e] / unit + 0.5);
    c = c < 1.0 ? 1.0 : c;
    c = c > (double)qmax ? (double)qmax : c;
    q[e] = (int32_t)c;
  }
}

// bounds for the gap sums (max of t * max(x, y)) and the line search (max of
// BPR(max(x, y)) * |y - x|)
__global__ void k_fw_bounds(const double* t0, const double* x, const unsigned* ycnt, const double* t,
                            const double* cap, double alpha, int beta, unsigned long long* out, int n) {
  double bg = 0.0, bl = 0.0;
  LS(e, n) {
    const double y = (double)ycnt[e];
    const double hi = x[e] > y ? x[e] : y;
    const double g = hi * t[e];
    const double l = bpr_t(t0[e], hi, cap[e], alpha, beta) * fabs(y - x[e]);
    bg = g > bg ? g : bg;
    bl = l > bl ? l : bl;
  }
  max_nonneg(&out[0], bg);
  max_nonneg(&out[1], bl);
}

__global__ void k_fw_gap_sums(const double* t, const double* x, const unsigned* ycnt, double scale,
                              unsigned long long* out, int n) {
  long long tx = 0, ty = 0;
  LS(e, n) {
    tx += __double2ll_rn(t[e] * x[e] * scale);
    ty += __double2ll_rn(t[e] * (double)ycnt[e] * scale);
  }
  add_fixed(&out[0], tx);
  add_fixed(&out[1], ty);
}

// derivative of the Beckmann objective along d = y - x at step a, on the fixed grid
__global__ void k_fw_deriv(const double* t0, const double* x, const unsigned* ycnt, const double* cap, double alpha,
                           int beta, double a, double scale, unsigned long long* out, int n) {
  long long g = 0;
  LS(e, n) {
    const double d = (double)ycnt[e] - x[e];
    g += __double2ll_rn(bpr_t(t0[e], x[e] + a * d, cap[e], alpha, beta) * d * scale);
  }
  add_fixed(out, g);
}

__global__ void k_fw_update(double* x, const unsigned* ycnt, double a, int n) {
  LS(e, n) x[e] = x[e] + a * ((double)ycnt[e] - x[e]);
}

__global__ void k_fw_obj_bound(const double* t0, const double* x, const double* cap, double alpha, int beta,
                               unsigned long long* out, int n) {
  double m = 0.0;
  LS(e, n) {
    const double f = bpr_area(t0[e], x[e], cap[e], alpha, beta);
    m = f > m ? f : m;
  }
  max_nonneg(out, m);
}

__global__ void k_fw_obj_sum(const double* t0, const double* x, const double* cap, double alpha, int beta,
                             double scale, unsigned long long* out, int n) {
  long long s = 0;
  LS(e, n) s += __double2ll_rn(bpr_area(t0[e], x[e], cap[e], alpha, beta) * scale);
  add_fixed(out, s);
}

__global__ void k_fw_final_time(const double* t0, const double* x, const double* cap, double alpha, int beta,
                                double* t, int n) {
  LS(e, n) t[e] = bpr_t(t0[e], x[e], cap[e], alpha, beta);
}

static int fw_grid(int n) {
  int g = (n + 255) / 256;
  return g < 1 ? 1 : (g > 2048 ? 2048 : g);
}

void launch_fw_t0(const float* len, const float* spd, double* t0, int n, cudaStream_t s) {
  k_fw_t0<<<fw_grid(n), 256, 0, s>>>(len, spd, t0, n);
}
void launch_fw_counts(const unsigned* cnt, double* x, int n, cudaStream_t s) {
  k_fw_counts<<<fw_grid(n), 256, 0, s>>>(cnt, x, n);
}
void launch_fw_time(const double* t0, const double* x, const double* cap, double alpha, int beta, double* t,
                    unsigned long long* tmax, int n, cudaStream_t s) {
  k_fw_time<<<fw_grid(n), 256, 0, s>>>(t0, x, cap, alpha, beta, t, tmax, n);
}
void launch_fw_quantize(const double* t, double unit, int qmax, int32_t* q, int n, cudaStream_t s) {
  k_fw_quantize<<<fw_grid(n), 256, 0, s>>>(t, unit, qmax, q, n);
}
void launch_fw_bounds(const double* t0, const double* x, const unsigned* y, const double* t, const double* cap,
                      double alpha, int beta, unsigned long long* out, int n, cudaStream_t s) {
  k_fw_bounds<<<fw_grid(n), 256, 0, s>>>(t0, x, y, t, cap, alpha, beta, out, n);
}
void launch_fw_gap_sums(const double* t, const double* x, const unsigned* y, double scale, unsigned long long* out,
                        int n, cudaStream_t s) {
  k_fw_gap_sums<<<fw_grid(n), 256, 0, s>>>(t, x, y, scale, out, n);
}
void launch_fw_deriv(const double* t0, const double* x, const unsigned* y, const double* cap, double alpha, int beta,
                     double a, double scale, unsigned long long* out, int n, cudaStream_t s) {
  k_fw_deriv<<<fw_grid(n), 256, 0, s>>>(t0, x, y, cap, alpha, beta, a, scale, out, n);
}
void launch_fw_update(double* x, const unsigned* y, double a, int n, cudaStream_t s) {
  k_fw_update<<<fw_grid(n), 256, 0, s>>>(x, y, a, n);
}
void launch_fw_objective(const double* t0, const double* x, const double* cap, double alpha, int beta, bool bound,
                         double scale, unsigned long long* out, int n, cudaStream_t s) {
  if (bound) k_fw_obj_bound<<<fw_grid(n), 256, 0, s>>>(t0, x, cap, alpha, beta, out, n);
  else k_fw_obj_sum<<<fw_grid(n), 256, 0, s>>>(t0, x, cap, alpha, beta, scale, out, n);
}
void launch_fw_final_time(const double* t0, const double* x, const double* cap, double alpha, int beta, double* t,
                          int n, cudaStream_t s) {
  k_fw_final_time<<<fw_grid(n), 256, 0, s>>>(t0, x, cap, alpha, beta, t, n);
}

}  // namespace gbt
