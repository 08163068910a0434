// Measured link travel times for the iterative decaying equilibrium (Waddell et al.,
// Sec. 6.3.1): after a run, each link's new routing weight is the mean of the
// traversal times recorded by the step kernels, in deciseconds, and the gap between
// the weights the run was routed on and the measured ones says how far the
// iteration is from travel times that reproduce themselves.
#include "gbt_internal.cuh"

namespace gbt {

// cost[e] = round_half_up(tt_sum[e] * dt_ds / tt_n[e]) within 1..1e6, or prev[e] when
// no trip left e.  Integer arithmetic throughout, so the result does not depend on
// the order of the atomics that built the sums.  The gap's numerator and denominator
// (sum n |cost - prev|, sum n prev) are added into ctl->gap_num / gap_den.
__global__ void k_measured_costs(Dev d, const int32_t* prev, int32_t* out) {
  unsigned long long num = 0, den = 0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.n_links; e += gridDim.x * blockDim.x) {
    const unsigned long long n = (unsigned long long)d.tt_n[e];
    const long long p = prev[e];
    if (n == 0) {
      out[e] = (int32_t)p;
      continue;
    }
    long long c = (long long)((2ULL * d.tt_sum[e] * (unsigned long long)d.dt_ds + n) / (2ULL * n));
    c = c < 1 ? 1 : (c > 1000000 ? 1000000 : c);
    out[e] = (int32_t)c;
    num += n * (unsigned long long)(c > p ? c - p : p - c);
    den += n * (unsigned long long)p;
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0 && (num | den)) {
    atomicAdd(&d.ctl->gap_num, num);
    atomicAdd(&d.ctl->gap_den, den);
  }
}

void launch_measured_costs(const Dev& d, const int32_t* prev, int32_t* out, cudaStream_t s) {
  int grid = (d.n_links + 255) / 256;
  if (grid > 1024) grid = 1024;
  if (grid < 1) grid = 1;
  k_measured_costs<<<grid, 256, 0, s>>>(d, prev, out);
}

}  // namespace gbt
