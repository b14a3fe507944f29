// Discrete adjoint of the explicit step (single-block cavity), FP64.
//
// Objective J = (1/N) sum_{n=1..N} Nu_hot(Q^n); controls: the hot-wall
// temperature field theta and Ra.  A step Q^{n+1} = G(Q^n) is: dt = cfl / S,
// S = max over nodes of the spectral bound of Q^n; Q~ = Q^n + dt R(Q^n)
// (Eqs. 1-3); p = p~ - mean of p~ over the centre nodes; walls formed from the
// new interior (Section 2) with the hot-wall temperature theta.  The reverse
// sweep over one step, given Xbar = dJ/dQ^{n+1} on the interior:
//   k_adj_objective  add dNu(Q^{n+1})/dQ^{n+1} / N (T next to the hot wall, theta)
//   k_adj_sum_p      sum of the p adjoint (the centre shift's transpose)
//   k_adj_prepare    Yt = Xbar minus that sum shared over the centre nodes;
//                    Q = Yt on the interior, 0 on walls and ghosts
//   k_adj_rates      at every interior node the reverse of the rates
//                    applied to dt Yt, added with FP64 atomics into Q at the
//                    stencil's inputs; sums of Yt R (for dt), of the
//                    buoyancy and beta^2-floor adjoints
//   k_adj_argmax + k_adj_dt  dt's dependence: -cfl dtbar / S^2 times the
//                    gradient of the spectral bound at its largest node
//   k_adj_fold       wall and ghost adjoints moved onto interior nodes 1, 2
//                    through p_w = 2 p1 - p2, p_g = 2 p_w - p1,
//                    T_w = (4 T1 - T2)/3, and the hot wall's T onto theta
//   k_adj_finish     Ra adjoint from the buoyancy (g sigma = Ra Pr) and floor
//                    (kappa u_ref^2 = kappa Ra Pr) sums; reset the scalars
// Subgradients at kinks follow the forward branch (|x| with sign(0) = 0, the
// beta^2 floor, the argmax node).  The state Q^n is read through the storage
// helpers, so the forward may be FP64 or FP32-mixed; the adjoint is FP64.
#pragma once

#include "bdc_device.cuh"

namespace bdc {

struct AdjGeom {  // dense FP64 adjoint arrays over local nodes -1 .. n+2, 5 fields
  int nx, ny, nz;
  long long ex, ey, fs;  // row length, rows, elements per field
};

__device__ __forceinline__ long long aidx(const AdjGeom &g, int f, int i, int j, int k) {
  return (long long)(i + 1) + g.ex * ((long long)(j + 1) + g.ey * (long long)(k + 1)) + g.fs * f;
}

enum { kScDtbar = 0, kScSumP = 1, kScGs = 2, kScFloor = 3, kScRa = 4, kScJ = 5, kScCount = 8 };

struct AdjArgs {
  BlockDev B;        // the state Q^n being read (buffer set base[0])
  CavConst C;
  AdjGeom g;
  double *X;         // adjoint of the interior state after the step
  double *Yt;        // X after the centre-shift transpose
  double *Q;         // scatter target: adjoint of Q^n (interior, walls, ghosts)
  double *scal;      // kSc* scalars
  double *thetabar;  // ny*nz, (j-1) + ny (k-1)
  double *argpart;   // per-CTA (max, index) pairs of k_adj_argmax
  double dt;         // dt of this step
  double coef;       // 1 / (N ny nz 2 h_x dT)
  double dfloor;     // d(beta^2 floor)/dRa
};

// state value of field f (0 = p, 1..4 = u, v, w, T) at local node (i, j, k)
template <class S>
__device__ __forceinline__ double st(const AdjArgs &a, int f, int i, int j, int k) {
  return get_field<S>((const S *)a.B.base[0], a.B.fstride, f, node_index<S>(a.B, i, j, k));
}

__global__ void k_adj_objective(AdjArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.g.ny * a.g.nz) return;
  const int j = e % a.g.ny + 1, k = e / a.g.ny + 1;
  a.X[aidx(a.g, 4, 1, j, k)] += -4.0 * a.coef;
  a.X[aidx(a.g, 4, 2, j, k)] += a.coef;
  a.thetabar[e] += 3.0 * a.coef;
}

__global__ void k_adj_sum_p(AdjArgs a) {
  const long long n = (long long)a.g.nx * a.g.ny * a.g.nz;
  double s = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % a.g.nx) + 1, j = (int)((e / a.g.nx) % a.g.ny) + 1, k = (int)(e / ((long long)a.g.nx * a.g.ny)) + 1;
    s += a.X[aidx(a.g, 0, i, j, k)];
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(&a.scal[kScSumP], s);
}

__global__ void k_adj_prepare(AdjArgs a) {
  const long long n = a.g.fs * 5;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int f = (int)(e / a.g.fs);
  const long long r = e % a.g.fs;
  const int i = (int)(r % a.g.ex) - 1, j = (int)((r / a.g.ex) % a.g.ey) - 1, k = (int)(r / (a.g.ex * a.g.ey)) - 1;
  double v = 0.0;
  if (i >= 1 && i <= a.g.nx && j >= 1 && j <= a.g.ny && k >= 1 && k <= a.g.nz) {
    v = a.X[e];
    if (f == 0) {
      const int *gn = a.C.gn;
      const bool ci = (gn[0] % 2) ? i == (gn[0] + 1) / 2 : (i == gn[0] / 2 || i == gn[0] / 2 + 1);
      const bool cj = (gn[1] % 2) ? j == (gn[1] + 1) / 2 : (j == gn[1] / 2 || j == gn[1] / 2 + 1);
      const bool ck = (gn[2] % 2) ? k == (gn[2] + 1) / 2 : (k == gn[2] / 2 || k == gn[2] / 2 + 1);
      if (ci && cj && ck) v -= a.scal[kScSumP] / (double)a.C.ncentre;
    }
  }
  a.Yt[e] = v;
  a.Q[e] = v;
}

// reverse of the rates at one interior node, scattered with atomics
template <class S>
__global__ void __launch_bounds__(256) k_adj_rates(AdjArgs a) {
  const long long n = (long long)a.g.nx * a.g.ny * a.g.nz;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double dtbar = 0.0, gsbar = 0.0, floorbar = 0.0;
  if (e < n) {
    const int i = (int)(e % a.g.nx) + 1, j = (int)((e / a.g.nx) % a.g.ny) + 1, k = (int)(e / ((long long)a.g.nx * a.g.ny)) + 1;
    const CavConst &C = a.C;
    const int o3[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    // stencil values: centre, then +d / -d per axis, and p at +-2d
    double c0[5], qp[5][3], qm[5][3], p2p[3], p2m[3];
    for (int f = 0; f < 5; ++f) c0[f] = st<S>(a, f, i, j, k);
    for (int d = 0; d < 3; ++d) {
      for (int f = 0; f < 5; ++f) {
        qp[f][d] = st<S>(a, f, i + o3[d][0], j + o3[d][1], k + o3[d][2]);
        qm[f][d] = st<S>(a, f, i - o3[d][0], j - o3[d][1], k - o3[d][2]);
      }
      p2p[d] = st<S>(a, 0, i + 2 * o3[d][0], j + 2 * o3[d][1], k + 2 * o3[d][2]);
      p2m[d] = st<S>(a, 0, i - 2 * o3[d][0], j - 2 * o3[d][1], k - 2 * o3[d][2]);
    }
    const double V[3] = {c0[1], c0[2], c0[3]};
    double b2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const bool floored = b2 < C.b2min;
    if (floored) b2 = C.b2min;
    double sq[3], lam[3], d4[3], a_[3], divV = 0.0, diss = 0.0;
    for (int d = 0; d < 3; ++d) {
      sq[d] = sqrt(V[d] * V[d] + 4.0 * b2);
      lam[d] = 0.5 * (fabs(V[d]) + sq[d]);
      d4[d] = (p2p[d] + p2m[d]) - 4.0 * (qp[0][d] + qm[0][d]) + 6.0 * c0[0];
      a_[d] = V[d] * C.ih2[d];
      divV += (qp[1 + d][d] - qm[1 + d][d]) * C.ih2[d];
      diss += C.c4 * lam[d] * C.ih[d] * d4[d];
    }
    // forward rates (for dt's adjoint: dtbar = sum Yt R)
    double R[5];
    R[0] = -b2 * divV - diss;
    for (int q = 1; q <= 4; ++q) {
      const double D = q == 4 ? C.alpha : C.nu;
      double r = 0.0;
      for (int d = 0; d < 3; ++d)
        r += (D * C.ihh[d] - a_[d]) * (qp[q][d] - c0[q]) + (D * C.ihh[d] + a_[d]) * (qm[q][d] - c0[q]);
      if (q <= 3) {
        const int cc = q - 1;
        r += -(qp[0][cc] - qm[0][cc]) * C.ih2[cc];
        if (cc == C.gaxis) r += C.gs * (c0[4] - C.t_inf);
      }
      R[q] = r;
    }
    double yt[5];
    for (int f = 0; f < 5; ++f) {
      yt[f] = a.Yt[aidx(a.g, f, i, j, k)];
      dtbar += yt[f] * R[f];
    }
    double rb[5];
    for (int f = 0; f < 5; ++f) rb[f] = a.dt * yt[f];
    // adjoints of the centre values (accumulated here, one atomic each at the end)
    double cbar[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    double abar[3] = {0.0, 0.0, 0.0};
    // transported fields
    for (int q = 1; q <= 4; ++q) {
      const double D = q == 4 ? C.alpha : C.nu;
      for (int d = 0; d < 3; ++d) {
        atomicAdd(&a.Q[aidx(a.g, q, i + o3[d][0], j + o3[d][1], k + o3[d][2])], rb[q] * (D * C.ihh[d] - a_[d]));
        atomicAdd(&a.Q[aidx(a.g, q, i - o3[d][0], j - o3[d][1], k - o3[d][2])], rb[q] * (D * C.ihh[d] + a_[d]));
        cbar[q] += -2.0 * rb[q] * D * C.ihh[d];
        abar[d] += -rb[q] * (qp[q][d] - qm[q][d]);
      }
      if (q <= 3) {
        const int cc = q - 1;
        atomicAdd(&a.Q[aidx(a.g, 0, i + o3[cc][0], j + o3[cc][1], k + o3[cc][2])], -rb[q] * C.ih2[cc]);
        atomicAdd(&a.Q[aidx(a.g, 0, i - o3[cc][0], j - o3[cc][1], k - o3[cc][2])], rb[q] * C.ih2[cc]);
        if (cc == C.gaxis) {
          cbar[4] += C.gs * rb[q];
          gsbar += (c0[4] - C.t_inf) * rb[q];
        }
      }
    }
    for (int d = 0; d < 3; ++d) cbar[1 + d] += abar[d] * C.ih2[d];
    // continuity: R_p = -b2 divV - diss
    double b2bar = -divV * rb[0];
    const double divbar = -b2 * rb[0], dissbar = -rb[0];
    for (int d = 0; d < 3; ++d) {
      atomicAdd(&a.Q[aidx(a.g, 1 + d, i + o3[d][0], j + o3[d][1], k + o3[d][2])], divbar * C.ih2[d]);
      atomicAdd(&a.Q[aidx(a.g, 1 + d, i - o3[d][0], j - o3[d][1], k - o3[d][2])], -divbar * C.ih2[d]);
      const double lambar = dissbar * C.c4 * C.ih[d] * d4[d];
      const double d4bar = dissbar * C.c4 * lam[d] * C.ih[d];
      atomicAdd(&a.Q[aidx(a.g, 0, i + 2 * o3[d][0], j + 2 * o3[d][1], k + 2 * o3[d][2])], d4bar);
      atomicAdd(&a.Q[aidx(a.g, 0, i - 2 * o3[d][0], j - 2 * o3[d][1], k - 2 * o3[d][2])], d4bar);
      atomicAdd(&a.Q[aidx(a.g, 0, i + o3[d][0], j + o3[d][1], k + o3[d][2])], -4.0 * d4bar);
      atomicAdd(&a.Q[aidx(a.g, 0, i - o3[d][0], j - o3[d][1], k - o3[d][2])], -4.0 * d4bar);
      cbar[0] += 6.0 * d4bar;
      const double sgn = V[d] > 0.0 ? 1.0 : (V[d] < 0.0 ? -1.0 : 0.0);
      cbar[1 + d] += lambar * 0.5 * (sgn + V[d] / sq[d]);
      b2bar += lambar / sq[d];
    }
    if (floored) {
      floorbar += b2bar;
    } else {
      for (int d = 0; d < 3; ++d) cbar[1 + d] += 2.0 * V[d] * b2bar;
    }
    for (int f = 0; f < 5; ++f) atomicAdd(&a.Q[aidx(a.g, f, i, j, k)], cbar[f]);
  }
  dtbar = warp_sum(dtbar);
  gsbar = warp_sum(gsbar);
  floorbar = warp_sum(floorbar);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&a.scal[kScDtbar], dtbar);
    atomicAdd(&a.scal[kScGs], gsbar);
    atomicAdd(&a.scal[kScFloor], floorbar);
  }
}

// largest spectral bound of Q^n and its node (smallest linear index among equal values)
template <class S>
__global__ void __launch_bounds__(256) k_adj_argmax(AdjArgs a) {
  const long long n = (long long)a.g.nx * a.g.ny * a.g.nz;
  double best = -1.0, bidx = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % a.g.nx) + 1, j = (int)((e / a.g.nx) % a.g.ny) + 1, k = (int)(e / ((long long)a.g.nx * a.g.ny)) + 1;
    const double s = spectral_f64(a.C, st<S>(a, 1, i, j, k), st<S>(a, 2, i, j, k), st<S>(a, 3, i, j, k));
    if (s > best) { best = s; bidx = (double)e; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o), oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
  }
  __shared__ double sb[8], si[8];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sb[w] = best; si[w] = bidx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
      if (sb[q] > best || (sb[q] == best && si[q] < bidx)) { best = sb[q]; bidx = si[q]; }
    a.argpart[2 * blockIdx.x] = best;
    a.argpart[2 * blockIdx.x + 1] = bidx;
  }
}

// dt = cfl / S: add (-cfl dtbar / S^2) d(bound)/dV at the argmax node (one thread)
template <class S>
__global__ void k_adj_dt(AdjArgs a, int nparts) {
  double best = -1.0, bidx = 0.0;
  for (int q = 0; q < nparts; ++q)
    if (a.argpart[2 * q] > best || (a.argpart[2 * q] == best && a.argpart[2 * q + 1] < bidx)) {
      best = a.argpart[2 * q];
      bidx = a.argpart[2 * q + 1];
    }
  const long long e = (long long)bidx;
  const int i = (int)(e % a.g.nx) + 1, j = (int)((e / a.g.nx) % a.g.ny) + 1, k = (int)(e / ((long long)a.g.nx * a.g.ny)) + 1;
  const double sbar = -a.C.cfl * a.scal[kScDtbar] / (best * best);
  const double V[3] = {st<S>(a, 1, i, j, k), st<S>(a, 2, i, j, k), st<S>(a, 3, i, j, k)};
  double b2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
  const bool floored = b2 < a.C.b2min;
  if (floored) b2 = a.C.b2min;
  double b2bar = 0.0, vbar[3];
  for (int d = 0; d < 3; ++d) {
    const double sq = sqrt(V[d] * V[d] + 4.0 * b2);
    const double sgn = V[d] > 0.0 ? 1.0 : (V[d] < 0.0 ? -1.0 : 0.0);
    vbar[d] = sbar * 0.5 * a.C.ih[d] * (sgn + V[d] / sq);
    b2bar += sbar * a.C.ih[d] / sq;
  }
  if (floored) a.scal[kScFloor] += b2bar;
  for (int d = 0; d < 3; ++d) a.Q[aidx(a.g, 1 + d, i, j, k)] += vbar[d] + (floored ? 0.0 : 2.0 * V[d] * b2bar);
}

// wall and ghost adjoints onto the interior nodes they are formed from
__global__ void k_adj_fold(AdjArgs a) {
  const int n[3] = {a.g.nx, a.g.ny, a.g.nz};
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int face = 0;
  for (; face < 6; ++face) {
    const int ax = face >> 1;
    const long long cnt = (long long)n[ax == 0 ? 1 : 0] * n[ax == 2 ? 1 : 2];
    if (e < cnt) break;
    e -= cnt;
  }
  if (face >= 6) return;
  const int ax = face >> 1, high = face & 1;
  const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
  const int c1 = (int)(e % n[a1]) + 1, c2 = (int)(e / n[a1]) + 1;
  const int w = high ? n[ax] + 1 : 0, s = high ? -1 : 1;
  int iw[3], i1[3], i2[3], ig[3];
  iw[ax] = w; i1[ax] = w + s; i2[ax] = w + 2 * s; ig[ax] = w - s;
  iw[a1] = i1[a1] = i2[a1] = ig[a1] = c1;
  iw[a2] = i1[a2] = i2[a2] = ig[a2] = c2;
  const double pw = a.Q[aidx(a.g, 0, iw[0], iw[1], iw[2])], pg = a.Q[aidx(a.g, 0, ig[0], ig[1], ig[2])];
  atomicAdd(&a.Q[aidx(a.g, 0, i1[0], i1[1], i1[2])], 2.0 * pw + 3.0 * pg);
  atomicAdd(&a.Q[aidx(a.g, 0, i2[0], i2[1], i2[2])], -pw - 2.0 * pg);
  const double tw = a.Q[aidx(a.g, 4, iw[0], iw[1], iw[2])];
  if (ax == 0) {
    if (!high) a.thetabar[(c1 - 1) + (long long)n[1] * (c2 - 1)] += tw;
  } else {
    atomicAdd(&a.Q[aidx(a.g, 4, i1[0], i1[1], i1[2])], (4.0 / 3.0) * tw);
    atomicAdd(&a.Q[aidx(a.g, 4, i2[0], i2[1], i2[2])], (-1.0 / 3.0) * tw);
  }
}

__global__ void k_adj_finish(AdjArgs a) {
  a.scal[kScRa] += a.C.nu * a.scal[kScGs] + a.dfloor * a.scal[kScFloor];
  a.scal[kScDtbar] = 0.0;
  a.scal[kScSumP] = 0.0;
  a.scal[kScGs] = 0.0;
  a.scal[kScFloor] = 0.0;
}

// J accumulation during the forward run: J += Nu_hot of cavity 0
__global__ void k_adj_acc_nusselt(const CavState *cs, double *scal) { scal[kScJ] += cs[0].nu_hot; }

}  // namespace bdc
