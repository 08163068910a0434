// Calibration adjoint of the step (not in the paper; the calibration workload of this
// library).  Loss L = sum over observations k and trips v of (p_v(t_k) - target)^2,
// p_v = route progress (completed link lengths + x; 0 before departure; the route's
// length after arrival).  The gradient with respect to every class's IDM parameters
// (v0, T, a, b, s0) holds the discrete decisions of the run fixed: the forward pass
// tapes, per vehicle-step, which form of Eq. 7 gave the acceleration (leader on the
// link, leader across the link end, free road, closed stop line), the gap and speeds
// that entered it, and how the ballistic move ended (normal, stopped within the step,
// clamped at the stop line, arrived).  The reverse sweep runs in binary64.
#include "gbt_internal.cuh"

namespace gbt {

#define GS(i, n) for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int ln = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (ln == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = ln < (int)(blockDim.x >> 5) ? sh[ln] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

__device__ __forceinline__ double prefix_len(const Dev& d, int vid, int upto) {
  const int off = d.roff[vid];
  double p = 0.0;
  for (int k = 0; k < upto; k++) p += (double)d.links[d.routes[off + k]].len;
  return p;
}

// Route progress of every trip at the current state (buffer A).  With target: the
// residual of the active trips goes to res (0 for the others, whose progress is
// constant) and the squared residuals of all trips are added to ctl->loss; with p_out:
// the progress itself.
__global__ void k_observe(Dev d, const double* target, double* res, double* p_out) {
  const int nA = d.ctl->nA;
  const int total = nA + d.n_trips;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int vid;
    double p;
    bool active;
    if (i < nA) {
      if (d.A.link[i] < 0) continue;
      vid = d.A.vid[i];
      p = prefix_len(d, vid, d.A.cur[i]) + (double)d.A.x[i];
      active = true;
    } else {
      vid = i - nA;
      const uint8_t st = d.status[vid];
      if (st == kActive) continue;
      p = st == kArrived ? prefix_len(d, vid, d.rlen[vid]) : 0.0;
      active = false;
    }
    if (p_out) p_out[vid] = p;
    if (target) {
      const double r = p - target[vid];
      acc += r * r;
      res[vid] = active ? r : 0.0;
    }
  }
  if (target) {
    const double b = block_sum(acc);
    if (threadIdx.x == 0) atomicAdd(&d.ctl->loss, b);
  }
}

void launch_observe(const Dev& d, int grid, cudaStream_t s, const double* target, double* res, double* p_out) {
  k_observe<<<grid, 256, 0, s>>>(d, target, res, p_out);
}

__global__ void k_tape_begin(Dev d) { d.ctl->tape_t0 = d.ctl->t; }

void launch_tape_begin(const Dev& d, cudaStream_t s) { k_tape_begin<<<1, 1, 0, s>>>(d); }

// Reverse of step t.  lx, lv: adjoint of the state after the step (by trip id), plus
// 2 * residual when that state was observed; nx, nv (zeroed): adjoint of the state
// before it.  Parameter gradients are summed per block in shared memory, then added.
__global__ void k_adj_step(Dev d, const TapeRec* slab, const double* lx, const double* lv, const double* res,
                           double* nx, double* nv, double* grad, int n_class) {
  extern __shared__ double sg[];
  for (int q = threadIdx.x; q < n_class * 5; q += blockDim.x) sg[q] = 0.0;
  __syncthreads();
  const double dt = d.dt, h = 0.5 * dt * dt;
  GS(i, d.n_trips) {
    const TapeRec r = slab[i];
    if (!r.valid) continue;
    const double lxp = lx[i] + (res ? 2.0 * res[i] : 0.0);
    const double lvp = lv[i];
    double mu = 0.0;
    if (r.branch == kBrNormal) {
      mu = lxp * h + lvp * dt;
      atomicAdd(&nx[i], lxp);
      atomicAdd(&nv[i], lxp * dt + lvp);
    } else if (r.branch == kBrStop) {
      const double a = r.a, v = r.v;
      mu = lxp * v * v / (2.0 * a * a);
      atomicAdd(&nx[i], lxp);
      atomicAdd(&nv[i], lxp * (-v / a));
    }
    if (mu == 0.0 || r.kind == kFormNone) continue;
    const LinkRec L = d.links[r.link];
    const ClassPar P = d.cls[L.cls];
    const double A = P.a, Bb = d.cls_b[L.cls], T = P.T, v0 = L.v0, v = r.v;
    const double rr = v / v0, r3 = rr * rr * rr, r4 = r3 * rr;
    double dA = 1.0 - r4, dv0 = 4.0 * A * r4 / v0, dv = -4.0 * A * r3 / v0;
    double ds = 0.0, dvl = 0.0, dT = 0.0, dB = 0.0, ds0 = 0.0;
    if (r.kind != kFormFree) {
      // the floors of Eq. 7, decided in binary32 exactly as the forward pass did
      const float dv32 = r.v - r.vl;
      const float t1 = r.v * P.T;
      const float t2 = (r.v * dv32) / P.sab2;
      const bool dyn_on = (t1 + t2) > 0.0f;
      const bool floored = !(r.s >= d.s_min) || r.s == d.s_min;
      const double vl = r.vl, s = r.s;
      const double cc = 1.0 / (2.0 * sqrt(A * Bb));
      const double dvv = v - vl;
      const double ss = (double)P.s0 + (dyn_on ? v * T + v * dvv * cc : 0.0);
      const double se = floored ? (double)d.s_min : s;
      const double q = ss / se;
      const double k2 = -2.0 * A * q / se;
      dA += -q * q;
      ds0 = k2;
      if (dyn_on) {
        dT = k2 * v;
        dA += k2 * v * dvv * (-cc / (2.0 * A));
        dB = k2 * v * dvv * (-cc / (2.0 * Bb));
        dv += k2 * (T + (dvv + v) * cc);
        dvl = k2 * (-v * cc);
      }
      ds = floored ? 0.0 : 2.0 * A * q * q / se;
      atomicAdd(&nx[i], -mu * ds);
      if (r.kind == kFormLead || r.kind == kFormNext) {
        atomicAdd(&nx[r.lead], mu * ds);
        atomicAdd(&nv[r.lead], mu * dvl);
      }
    }
    atomicAdd(&nv[i], mu * dv);
    const int c = L.cls;
    if (d.cls_v0_param[c]) atomicAdd(&sg[c * 5 + 0], mu * dv0);
    atomicAdd(&sg[c * 5 + 1], mu * dT);
    atomicAdd(&sg[c * 5 + 2], mu * dA);
    atomicAdd(&sg[c * 5 + 3], mu * dB);
    atomicAdd(&sg[c * 5 + 4], mu * ds0);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n_class * 5; q += blockDim.x)
    if (sg[q] != 0.0) atomicAdd(&grad[q], sg[q]);
}

void launch_adj_step(const Dev& d, int grid, cudaStream_t s, const TapeRec* slab, const double* lx,
                     const double* lv, const double* res, double* nx, double* nv, double* grad, int n_class) {
  k_adj_step<<<grid, 256, (size_t)n_class * 5 * sizeof(double), s>>>(d, slab, lx, lv, res, nx, nv, grad, n_class);
}

}  // namespace gbt
