// Discrete adjoint of the explicit step (single-block cavity).
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
//                    applied to dt Yt, added with atomics into Q at the
//                    stencil's inputs; sums of Yt R (for dt), of the
//                    buoyancy and beta^2-floor adjoints
//     (FP32 sweep instead: k_adj_pre does the objective, the sum and, in its
//     last CTA, the centre correction to Xbar in place; k_adj_gather reads
//     Xbar as Yt and writes every Q once, gathering what the stencils would
//     scatter; its node sums go out as per-CTA partials)
//   k_adj_argmax + k_adj_dt  dt's dependence: -cfl dtbar / S^2 times the
//                    gradient of the spectral bound at its largest node (the
//                    FP32 bound f32_spectral_exact after an FP32-mixed forward,
//                    which sets that forward's dt; the FP32 sweep takes the
//                    argmax of a whole recomputed segment in one launch,
//                    k_adj_argmax_seg); then the Ra adjoint from the buoyancy
//                    (g sigma = Ra Pr) and floor (kappa u_ref^2 = kappa Ra
//                    Pr) sums, and the per-step scalars reset
//   k_adj_fold       wall and ghost adjoints moved onto interior nodes 1, 2
//                    through p_w = 2 p1 - p2, p_g = 2 p_w - p1,
//                    T_w = (4 T1 - T2)/3, and the hot wall's T onto theta
// Subgradients at kinks follow the forward branch (|x| with sign(0) = 0, the
// beta^2 floor, the argmax node).
//
// Precision: the adjoint arrays X, Yt, Q hold A (the reverse sweep's type):
// FP64 after an FP64 forward, FP32 after an FP32-mixed forward, whose
// trajectory carries FP32 precision anyway.  The rates' reverse works on
// neighbour-minus-centre differences; for the FP32-mixed state the p and T
// differences are formed from their hi/lo pairs (as the forward step does),
// so FP32 arithmetic loses no cancellation.  The sums over nodes (dt, g sigma,
// beta^2 floor, the p adjoint) are FP64 beyond a warp (the FP32 sweep adds at
// most a few dozen terms in FP32 per lane or warp first); the wall gradient
// stays FP64.
#pragma once

#include <type_traits>

#include "bdc_device.cuh"
#include "bdc_step_f32.cuh"

namespace bdc {

struct AdjGeom {  // dense adjoint arrays over local nodes -1 .. n+2, 5 fields
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
  void *X;           // adjoint of the interior state after the step (type A)
  void *Yt;          // X after the centre-shift transpose (type A)
  void *Q;           // scatter target: adjoint of Q^n, interior, walls, ghosts (type A)
  double *scal;      // kSc* scalars
  double *thetabar;  // ny*nz, (j-1) + ny (k-1)
  double *argpart;   // per-CTA (max, index) pairs of k_adj_argmax
  double *gpart;     // per-CTA (dtbar, g sigma bar, floor bar) sums of k_adj_gather
  double *gpart2;    // the same, summed over contiguous runs of gpart by k_adj_argmax's CTAs
  int ngpart;        // k_adj_gather CTAs (0: the sums go to scal by atomics, k_adj_rates)
  double dt;         // dt of this step
  double coef;       // 1 / (N ny nz 2 h_x dT)
  double dfloor;     // d(beta^2 floor)/dRa
};

template <class A> __device__ __forceinline__ A *arr(void *p) { return static_cast<A *>(p); }

// interior node (i, j, k), 1-based, of linear interior index e (x fastest);
// 32-bit division: the adjoint's block has fewer than 2^31 interior nodes
__device__ __forceinline__ void unflat(const AdjGeom &g, unsigned e, int &i, int &j, int &k) {
  const unsigned nx = (unsigned)g.nx, ny = (unsigned)g.ny;
  const unsigned r = e / nx;
  i = (int)(e - r * nx) + 1;
  j = (int)(r % ny) + 1;
  k = (int)(r / ny) + 1;
}

// state value of field f (0 = p, 1..4 = u, v, w, T) at local node (i, j, k)
template <class S>
__device__ __forceinline__ double st(const AdjArgs &a, int f, int i, int j, int k) {
  return get_field<S>((const S *)a.B.base[0], a.B.fstride, f, node_index<S>(a.B, i, j, k));
}

template <class A>
__global__ void k_adj_objective(AdjArgs a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.g.ny * a.g.nz) return;
  const int j = e % a.g.ny + 1, k = e / a.g.ny + 1;
  A *X = arr<A>(a.X);
  X[aidx(a.g, 4, 1, j, k)] += (A)(-4.0 * a.coef);
  X[aidx(a.g, 4, 2, j, k)] += (A)a.coef;
  a.thetabar[e] += 3.0 * a.coef;
}

template <class A>
__global__ void __launch_bounds__(256) k_adj_sum_p(AdjArgs a) {
  // a warp per interior row (j, k), strided over the grid's warps: no index
  // division; each lane sums its values in A (the sweep's type), the warp
  // and the CTA in FP64, one atomic per CTA
  const A *X = arr<A>(a.X);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rows = a.g.ny * a.g.nz;
  A s = 0;
  for (int r = blockIdx.x * nw + w; r < rows; r += gridDim.x * nw) {
    const A *row = X + aidx(a.g, 0, 0, r % a.g.ny + 1, r / a.g.ny + 1);
    for (int i = 1 + lane; i <= a.g.nx; i += 32) s += row[i];
  }
  double d = warp_sum((double)s);
  __shared__ double red[8];
  if (lane == 0) red[w] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < nw; ++q) d += red[q];
    atomicAdd(&a.scal[kScSumP], d);
  }
}

// The FP32 sweep's first kernel of a reverse step, three steps in one: the
// objective's terms (as k_adj_objective), the sum of the p adjoint (as
// k_adj_sum_p, one FP64 atomic per CTA), and, in the CTA that finishes last,
// the centre-shift transpose in place (as k_adj_centre).  The objective
// touches T only and the sum reads p only, so the two share no data; `cnt`
// counts the finished CTAs (zero between launches).
template <class A>
__global__ void __launch_bounds__(256) k_adj_pre(AdjArgs a, unsigned int *cnt) {
  A *X = arr<A>(a.X);
  const int tid = threadIdx.x;
  for (int e = blockIdx.x * blockDim.x + tid; e < a.g.ny * a.g.nz; e += gridDim.x * blockDim.x) {
    const int j = e % a.g.ny + 1, k = e / a.g.ny + 1;
    X[aidx(a.g, 4, 1, j, k)] += (A)(-4.0 * a.coef);
    X[aidx(a.g, 4, 2, j, k)] += (A)a.coef;
    a.thetabar[e] += 3.0 * a.coef;
  }
  const int lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const int rows = a.g.ny * a.g.nz;
  A s = 0;
  for (int r = blockIdx.x * nw + w; r < rows; r += gridDim.x * nw) {
    const A *row = X + aidx(a.g, 0, 0, r % a.g.ny + 1, r / a.g.ny + 1);
    for (int i = 1 + lane; i <= a.g.nx; i += 32) s += row[i];
  }
  double d = warp_sum((double)s);
  __shared__ double red[8];
  __shared__ bool last;
  if (lane == 0) red[w] = d;
  __syncthreads();
  if (tid == 0) {
    for (int q = 1; q < nw; ++q) d += red[q];
    atomicAdd(&a.scal[kScSumP], d);
    __threadfence();
    last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (tid < 8) {
    int x[3];
    for (int dd = 0; dd < 3; ++dd) {
      const int n = a.C.gn[dd], up = (tid >> dd) & 1;
      if ((n % 2) && up) return;
      x[dd] = (n % 2) ? (n + 1) / 2 : n / 2 + up;
    }
    const long long e = aidx(a.g, 0, x[0], x[1], x[2]);
    X[e] = (A)((double)X[e] - __ldcg(&a.scal[kScSumP]) / (double)a.C.ncentre);
  }
  if (tid == 0) *cnt = 0u;
}

// The centre-shift transpose in place, for the gather sweep: X(p) at the
// (at most 8) centre nodes less sum_p / ncentre; everywhere else Yt = X on
// the interior, and the gather never uses a value off the interior.  One
// thread per centre node: bit d of the thread index picks the upper of two
// centre indices along axis d (threads whose axis has one centre index
// with the bit set return).
template <class A>
__global__ void k_adj_centre(AdjArgs a) {
  const int t = threadIdx.x;
  int x[3];
  for (int d = 0; d < 3; ++d) {
    const int n = a.C.gn[d], up = (t >> d) & 1;
    if ((n % 2) && up) return;
    x[d] = (n % 2) ? (n + 1) / 2 : n / 2 + up;
  }
  A *X = arr<A>(a.X);
  const long long e = aidx(a.g, 0, x[0], x[1], x[2]);
  X[e] = (A)((double)X[e] - a.scal[kScSumP] / (double)a.C.ncentre);
}

// Grid: x over the padded nodes of one field (fewer than 2^31: 32-bit index
// arithmetic), y over the five fields.  WQ: also initialise the scatter
// target Q (k_adj_rates adds into it; k_adj_gather writes every Q itself).
template <class A, bool WQ>
__global__ void k_adj_prepare(AdjArgs a) {
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= (unsigned)a.g.fs) return;
  const int f = blockIdx.y;
  const long long e = (long long)f * a.g.fs + r;
  const unsigned ex = (unsigned)a.g.ex, ey = (unsigned)a.g.ey, rq = r / ex;
  const int i = (int)(r - rq * ex) - 1, j = (int)(rq % ey) - 1, k = (int)(rq / ey) - 1;
  A v = 0;
  if (i >= 1 && i <= a.g.nx && j >= 1 && j <= a.g.ny && k >= 1 && k <= a.g.nz) {
    v = arr<A>(a.X)[e];
    if (f == 0) {
      const int *gn = a.C.gn;
      const bool ci = (gn[0] % 2) ? i == (gn[0] + 1) / 2 : (i == gn[0] / 2 || i == gn[0] / 2 + 1);
      const bool cj = (gn[1] % 2) ? j == (gn[1] + 1) / 2 : (j == gn[1] / 2 || j == gn[1] / 2 + 1);
      const bool ck = (gn[2] % 2) ? k == (gn[2] + 1) / 2 : (k == gn[2] / 2 || k == gn[2] / 2 + 1);
      if (ci && cj && ck) v = (A)((double)v - a.scal[kScSumP] / (double)a.C.ncentre);
    }
  }
  arr<A>(a.Yt)[e] = v;
  if (WQ) arr<A>(a.Q)[e] = v;
}

// The node's stencil as the reverse of the rates needs it: the velocities,
// neighbour-minus-centre differences dp[f][d] (node + e_d) and dm[f][d]
// (node - e_d) of the five fields, p's at +-2 e_d, and tb = T - T_inf.
template <class R>
struct AdjStencil {
  R V[3], dp[5][3], dm[5][3], d2p[3], d2m[3], tb;
};

template <class S, class R>
__device__ __forceinline__ void load_stencil(const AdjArgs &a, int i, int j, int k, AdjStencil<R> &s) {
  const int o3[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  if constexpr (std::is_same<S, float>::value && std::is_same<R, float>::value) {
    // FP32-mixed state: p and T as hi/lo pairs, differences formed per part
    const float *q = (const float *)a.B.base[0];
    const long long fs = a.B.fstride, o = node_index<float>(a.B, i, j, k);
    const long long step[3] = {1, a.B.pitch, a.B.plane};
    const float ph = q[o], pl = q[fs + o], th = q[5 * fs + o], tl = q[6 * fs + o];
    const float c[3] = {q[2 * fs + o], q[3 * fs + o], q[4 * fs + o]};
    auto pdf = [&](long long off) { return (q[o + off] - ph) + (q[fs + o + off] - pl); };
    auto tdf = [&](long long off) { return (q[5 * fs + o + off] - th) + (q[6 * fs + o + off] - tl); };
    for (int d = 0; d < 3; ++d) {
      const long long st_ = step[d];
      s.V[d] = c[d];
      s.dp[0][d] = pdf(st_);
      s.dm[0][d] = pdf(-st_);
      s.d2p[d] = pdf(2 * st_);
      s.d2m[d] = pdf(-2 * st_);
      for (int f = 1; f <= 3; ++f) {
        s.dp[f][d] = q[(1 + f) * fs + o + st_] - c[f - 1];
        s.dm[f][d] = q[(1 + f) * fs + o - st_] - c[f - 1];
      }
      s.dp[4][d] = tdf(st_);
      s.dm[4][d] = tdf(-st_);
    }
    s.tb = (th - (float)a.C.t_inf) + tl;
  } else {
    double c0[5];
    for (int f = 0; f < 5; ++f) c0[f] = st<S>(a, f, i, j, k);
    for (int d = 0; d < 3; ++d) {
      s.V[d] = (R)c0[1 + d];
      for (int f = 0; f < 5; ++f) {
        s.dp[f][d] = (R)(st<S>(a, f, i + o3[d][0], j + o3[d][1], k + o3[d][2]) - c0[f]);
        s.dm[f][d] = (R)(st<S>(a, f, i - o3[d][0], j - o3[d][1], k - o3[d][2]) - c0[f]);
      }
      s.d2p[d] = (R)(st<S>(a, 0, i + 2 * o3[d][0], j + 2 * o3[d][1], k + 2 * o3[d][2]) - c0[0]);
      s.d2m[d] = (R)(st<S>(a, 0, i - 2 * o3[d][0], j - 2 * o3[d][1], k - 2 * o3[d][2]) - c0[0]);
    }
    s.tb = (R)(c0[4] - a.C.t_inf);
  }
}

__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }

// Reverse of the rates at one interior node in type R, scattered with atomics
// into Q (type R).  The forward rates are formed from the same differences,
// since 4th differences and gradients need only neighbour-minus-centre values.
template <class S, class R>
__global__ void __launch_bounds__(256) k_adj_rates(AdjArgs a) {
  const long long n = (long long)a.g.nx * a.g.ny * a.g.nz;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double dtbar = 0.0, gsbar = 0.0, floorbar = 0.0;
  if (e < n) {
    int i, j, k;
    unflat(a.g, (unsigned)e, i, j, k);
    const CavConst &C = a.C;
    const int o3[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    R *Q = arr<R>(a.Q);
    AdjStencil<R> s;
    load_stencil<S, R>(a, i, j, k, s);
    const R *V = s.V;
    const R ih[3] = {(R)C.ih[0], (R)C.ih[1], (R)C.ih[2]}, ih2[3] = {(R)C.ih2[0], (R)C.ih2[1], (R)C.ih2[2]};
    const R ihh[3] = {(R)C.ihh[0], (R)C.ihh[1], (R)C.ihh[2]};
    const R c4 = (R)C.c4, nu = (R)C.nu, alpha = (R)C.alpha, gs = (R)C.gs;
    R b2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const bool floored = b2 < (R)C.b2min;
    if (floored) b2 = (R)C.b2min;
    // sq = sqrt(V_d^2 + 4 b2) and isq = 1/sq from one reciprocal square root
    // (the reverse needs V_d / sq and 1 / sq: no divisions)
    R sq[3], isq[3], lam[3], d4[3], ad[3], divV = 0, diss = 0;
    for (int d = 0; d < 3; ++d) {
      const R qd = V[d] * V[d] + (R)4 * b2;
      isq[d] = rsqrt_r(qd);
      sq[d] = qd * isq[d];
      lam[d] = (R)0.5 * ((V[d] < 0 ? -V[d] : V[d]) + sq[d]);
      d4[d] = (s.d2p[d] + s.d2m[d]) - (R)4 * (s.dp[0][d] + s.dm[0][d]);
      ad[d] = V[d] * ih2[d];
      divV += (s.dp[1 + d][d] - s.dm[1 + d][d]) * ih2[d];
      diss += c4 * lam[d] * ih[d] * d4[d];
    }
    // forward rates (for dt's adjoint: dtbar = sum Yt R)
    R Rf[5];
    Rf[0] = -b2 * divV - diss;
    for (int q = 1; q <= 4; ++q) {
      const R D = q == 4 ? alpha : nu;
      R r = 0;
      for (int d = 0; d < 3; ++d) r += (D * ihh[d] - ad[d]) * s.dp[q][d] + (D * ihh[d] + ad[d]) * s.dm[q][d];
      if (q <= 3) {
        const int cc = q - 1;
        r += -(s.dp[0][cc] - s.dm[0][cc]) * ih2[cc];
        if (cc == C.gaxis) r += gs * s.tb;
      }
      Rf[q] = r;
    }
    const R *Yt = arr<R>(a.Yt);
    R yt[5], dtb = 0;
    for (int f = 0; f < 5; ++f) {
      yt[f] = Yt[aidx(a.g, f, i, j, k)];
      dtb += yt[f] * Rf[f];
    }
    dtbar = (double)dtb;
    R rb[5];
    for (int f = 0; f < 5; ++f) rb[f] = (R)a.dt * yt[f];
    // adjoints of the centre values (accumulated here, one atomic each at the end)
    R cbar[5] = {0, 0, 0, 0, 0};
    R abar[3] = {0, 0, 0};
    R gsb = 0;
    // transported fields
    for (int q = 1; q <= 4; ++q) {
      const R D = q == 4 ? alpha : nu;
      for (int d = 0; d < 3; ++d) {
        atomicAdd(&Q[aidx(a.g, q, i + o3[d][0], j + o3[d][1], k + o3[d][2])], rb[q] * (D * ihh[d] - ad[d]));
        atomicAdd(&Q[aidx(a.g, q, i - o3[d][0], j - o3[d][1], k - o3[d][2])], rb[q] * (D * ihh[d] + ad[d]));
        cbar[q] += (R)(-2) * rb[q] * D * ihh[d];
        abar[d] += -rb[q] * (s.dp[q][d] - s.dm[q][d]);
      }
      if (q <= 3) {
        const int cc = q - 1;
        atomicAdd(&Q[aidx(a.g, 0, i + o3[cc][0], j + o3[cc][1], k + o3[cc][2])], -rb[q] * ih2[cc]);
        atomicAdd(&Q[aidx(a.g, 0, i - o3[cc][0], j - o3[cc][1], k - o3[cc][2])], rb[q] * ih2[cc]);
        if (cc == C.gaxis) {
          cbar[4] += gs * rb[q];
          gsb += s.tb * rb[q];
        }
      }
    }
    gsbar = (double)gsb;
    for (int d = 0; d < 3; ++d) cbar[1 + d] += abar[d] * ih2[d];
    // continuity: R_p = -b2 divV - diss
    R b2bar = -divV * rb[0];
    const R divbar = -b2 * rb[0], dissbar = -rb[0];
    for (int d = 0; d < 3; ++d) {
      atomicAdd(&Q[aidx(a.g, 1 + d, i + o3[d][0], j + o3[d][1], k + o3[d][2])], divbar * ih2[d]);
      atomicAdd(&Q[aidx(a.g, 1 + d, i - o3[d][0], j - o3[d][1], k - o3[d][2])], -divbar * ih2[d]);
      const R lambar = dissbar * c4 * ih[d] * d4[d];
      const R d4bar = dissbar * c4 * lam[d] * ih[d];
      atomicAdd(&Q[aidx(a.g, 0, i + 2 * o3[d][0], j + 2 * o3[d][1], k + 2 * o3[d][2])], d4bar);
      atomicAdd(&Q[aidx(a.g, 0, i - 2 * o3[d][0], j - 2 * o3[d][1], k - 2 * o3[d][2])], d4bar);
      atomicAdd(&Q[aidx(a.g, 0, i + o3[d][0], j + o3[d][1], k + o3[d][2])], (R)(-4) * d4bar);
      atomicAdd(&Q[aidx(a.g, 0, i - o3[d][0], j - o3[d][1], k - o3[d][2])], (R)(-4) * d4bar);
      cbar[0] += (R)6 * d4bar;
      const R sgn = V[d] > 0 ? (R)1 : (V[d] < 0 ? (R)(-1) : (R)0);
      cbar[1 + d] += lambar * (R)0.5 * (sgn + V[d] * isq[d]);
      b2bar += lambar * isq[d];
    }
    if (floored) {
      floorbar = (double)b2bar;
    } else {
      for (int d = 0; d < 3; ++d) cbar[1 + d] += (R)2 * V[d] * b2bar;
    }
    for (int f = 0; f < 5; ++f) atomicAdd(&Q[aidx(a.g, f, i, j, k)], cbar[f]);
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

// Gather form of k_adj_rates for the FP32 sweep (FP32-mixed state): one
// thread per node m of the padded arrays (walls and ghosts included) sums
// what the interior nodes of its stencil would have scattered into it --
// recomputing their coefficients from their velocities and Yt -- adds its
// own centre terms when m is interior, and writes Q(m) once: no atomics.
// Q(m) = Yt(m) + sum of incoming contributions (Yt is zero off the interior).
__global__ void __launch_bounds__(256) k_adj_gather(AdjArgs a) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float dtbsum = 0.f, gsbsum = 0.f, flbsum = 0.f;
  if (e < a.g.fs) {
    // (i, j, k) from the padded linear index: 32-bit arithmetic (fewer than
    // 2^31 padded nodes; 64-bit division is a long software sequence)
    const unsigned r = (unsigned)e, ex = (unsigned)a.g.ex, ey = (unsigned)a.g.ey, rq = r / ex;
    const int i = (int)(r - rq * ex) - 1, j = (int)(rq % ey) - 1, k = (int)(rq / ey) - 1;
    const CavConst &C = a.C;
    const float *q = (const float *)a.B.base[0];
    const long long fs = a.B.fstride;
    const float *Yt = arr<float>(a.Yt);
    const float dt = (float)a.dt;
    // FP32 constants rounded on the host (no per-thread conversions)
    const float ih[3] = {C.fih[0], C.fih[1], C.fih[2]};
    const float ih2[3] = {C.fh2[0], C.fh2[1], C.fh2[2]};
    const float ihh[3] = {C.fihh[0], C.fihh[1], C.fihh[2]};
    const float c4 = C.fc4, b2min = C.fb2min, Dq[5] = {0.f, C.fnu, C.fnu, C.fnu, C.falpha};
    const int nn[3] = {a.g.nx, a.g.ny, a.g.nz};
    auto interior = [&](int x, int y, int z) { return x >= 1 && x <= nn[0] && y >= 1 && y <= nn[1] && z >= 1 && z <= nn[2]; };
    float out[5];
    const bool inner = interior(i, j, k);
    for (int f = 0; f < 5; ++f) out[f] = inner ? Yt[aidx(a.g, f, i, j, k)] : 0.f;
    auto lambda = [&](float Vd, float b2) {
      const float qd = Vd * Vd + 4.f * b2;
      return 0.5f * (fabsf(Vd) + qd * rsqrtf(qd));
    };
    // Sources n = m + s e_d and m + 2 s e_d.  Every load is unconditional
    // (at n when n is interior, else at m, which is always in range), so the
    // loads issue together; a select drops the contributions of non-interior n.
    // Offsets in 32 bits: both the adjoint arrays (5 fs) and the state (7
    // fstride) have fewer than 2^31 elements.
    const int astr[3] = {1, (int)a.g.ex, (int)(a.g.ex * a.g.ey)};
    const int sstr[3] = {1, a.B.pitch, (int)a.B.plane};
    const int om = (int)node_index<float>(a.B, i, j, k);
    const int ei = (int)e, fsa = (int)a.g.fs, fs32 = (int)fs;
    const int xm[3] = {i, j, k};
    for (int d = 0; d < 3; ++d) {
      for (int s = -1; s <= 1; s += 2) {
        // first neighbour: transport, pressure gradient, divergence, dissipation (-4 d4bar at n +- e_d)
        {
          const int c = xm[d] + s;
          int x3[3] = {i, j, k};
          x3[d] = c;
          const bool in = interior(x3[0], x3[1], x3[2]);
          const int ea = in ? ei + s * astr[d] : ei, es = in ? om + s * sstr[d] : om;
          const float V[3] = {q[2 * fs32 + es], q[3 * fs32 + es], q[4 * fs32 + es]};
          const float b2 = fmaxf(V[0] * V[0] + V[1] * V[1] + V[2] * V[2], b2min);
          float rb[5];
          for (int f = 0; f < 5; ++f) rb[f] = dt * Yt[ea + f * fsa];
          const float ad = V[d] * ih2[d];
          for (int f = 1; f <= 4; ++f) {
            const float cf = rb[f] * (Dq[f] * ihh[d] + (float)s * ad);
            out[f] += in ? cf : 0.f;
          }
          float c0 = (float)s * rb[1 + d] * ih2[d] + 4.f * rb[0] * c4 * lambda(V[d], b2) * ih[d];
          float c1 = (float)s * b2 * rb[0] * ih2[d];  // -s divbar ih2, divbar = -b2 rb0
          out[0] += in ? c0 : 0.f;
          out[1 + d] += in ? c1 : 0.f;
        }
        // second neighbour: dissipation (d4bar at n +- 2 e_d), d4bar = -rb0 c4 lambda ih
        {
          int x3[3] = {i, j, k};
          x3[d] = xm[d] + 2 * s;
          const bool in = interior(x3[0], x3[1], x3[2]);
          const int ea = in ? ei + 2 * s * astr[d] : ei, es = in ? om + 2 * s * sstr[d] : om;
          const float V[3] = {q[2 * fs32 + es], q[3 * fs32 + es], q[4 * fs32 + es]};
          const float b2 = fmaxf(V[0] * V[0] + V[1] * V[1] + V[2] * V[2], b2min);
          const float c0 = -dt * Yt[ea] * c4 * lambda(V[d], b2) * ih[d];
          out[0] += in ? c0 : 0.f;
        }
      }
    }
    if (inner) {
      // centre terms of m itself (the diagonal of the node's own reverse) and
      // the node sums, as in k_adj_rates
      AdjStencil<float> st_;
      load_stencil<float, float>(a, i, j, k, st_);
      const float *V = st_.V;
      float b2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
      const bool floored = b2 < b2min;
      if (floored) b2 = b2min;
      float sq[3], isq[3], lam[3], d4[3], ad[3], divV = 0.f, diss = 0.f;
      for (int d = 0; d < 3; ++d) {
        const float qd = V[d] * V[d] + 4.f * b2;
        isq[d] = rsqrtf(qd);
        sq[d] = qd * isq[d];
        lam[d] = 0.5f * (fabsf(V[d]) + sq[d]);
        d4[d] = (st_.d2p[d] + st_.d2m[d]) - 4.f * (st_.dp[0][d] + st_.dm[0][d]);
        ad[d] = V[d] * ih2[d];
        divV += (st_.dp[1 + d][d] - st_.dm[1 + d][d]) * ih2[d];
        diss += c4 * lam[d] * ih[d] * d4[d];
      }
      float Rf[5];
      Rf[0] = -b2 * divV - diss;
      for (int f = 1; f <= 4; ++f) {
        float r = 0.f;
        for (int d = 0; d < 3; ++d) r += (Dq[f] * ihh[d] - ad[d]) * st_.dp[f][d] + (Dq[f] * ihh[d] + ad[d]) * st_.dm[f][d];
        if (f <= 3) {
          const int cc = f - 1;
          r += -(st_.dp[0][cc] - st_.dm[0][cc]) * ih2[cc];
          if (cc == C.gaxis) r += C.fgs * st_.tb;
        }
        Rf[f] = r;
      }
      float yt[5], rb[5], dtb = 0.f;
      for (int f = 0; f < 5; ++f) {
        yt[f] = Yt[aidx(a.g, f, i, j, k)];
        dtb += yt[f] * Rf[f];
        rb[f] = dt * yt[f];
      }
      dtbsum = dtb;
      float abar[3] = {0.f, 0.f, 0.f}, gsb = 0.f;
      for (int f = 1; f <= 4; ++f) {
        for (int d = 0; d < 3; ++d) {
          out[f] += -2.f * rb[f] * Dq[f] * ihh[d];
          abar[d] += -rb[f] * (st_.dp[f][d] - st_.dm[f][d]);
        }
        if (f <= 3 && f - 1 == C.gaxis) {
          out[4] += C.fgs * rb[f];
          gsb += st_.tb * rb[f];
        }
      }
      gsbsum = gsb;
      for (int d = 0; d < 3; ++d) out[1 + d] += abar[d] * ih2[d];
      float b2bar = -divV * rb[0];
      for (int d = 0; d < 3; ++d) {
        const float lambar = -rb[0] * c4 * ih[d] * d4[d];
        out[0] += 6.f * (-rb[0] * c4 * lam[d] * ih[d]);
        const float sgn = V[d] > 0.f ? 1.f : (V[d] < 0.f ? -1.f : 0.f);
        out[1 + d] += lambar * 0.5f * (sgn + V[d] * isq[d]);
        b2bar += lambar * isq[d];
      }
      if (floored) {
        flbsum = b2bar;
      } else {
        for (int d = 0; d < 3; ++d) out[1 + d] += 2.f * V[d] * b2bar;
      }
    }
    float *Q = arr<float>(a.Q);
    for (int f = 0; f < 5; ++f) Q[aidx(a.g, f, i, j, k)] = out[f];
  }
  // node sums: FP32 within a warp (32 terms), FP64 across the CTA's warps,
  // one partial per CTA (no same-address atomics; k_adj_dt reduces the
  // partials in a fixed order)
  float s3[3] = {dtbsum, gsbsum, flbsum};
  for (int q = 0; q < 3; ++q) s3[q] = warp_sum_f(s3[q]);
  __shared__ double red[256 / 32][3];
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 3; ++q) red[threadIdx.x >> 5][q] = (double)s3[q];
  __syncthreads();
  if (threadIdx.x < 3) {
    double acc = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += red[w][threadIdx.x];
    a.gpart[3 * (long long)blockIdx.x + threadIdx.x] = acc;
  }
}

// Largest spectral bound of the state in buffer set 0 of block B and its
// node (smallest linear index among equal values: each thread visits its
// nodes in increasing index), over the rows of CTA `cta` of `ncta`; thread 0
// writes (max, index) to out2.  Every thread of the CTA calls it.
template <class S>
__device__ __forceinline__ void adj_argmax_part(const BlockDev &B, const CavConst &C, const AdjGeom &g, int cta, int ncta,
                                                double *out2) {
  // a warp per interior row (j, k), strided over the grid's warps (no index
  // division); a thread visits its nodes in increasing linear interior index
  // e = (i - 1) + nx ((j - 1) + ny (k - 1)), so it keeps the first of equal values
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5, nwq = blockDim.x >> 5;
  const int nx = g.nx, ny = g.ny, rows = ny * g.nz;
  const S *q = (const S *)B.base[0];
  const long long fs = B.fstride;
  constexpr int NP = Store<S>::NP;  // u, v, w follow the p array(s)
  double best = -1.0, bidx = 0.0;
  float bestf = -1.f;               // FP32 path: the running maximum in FP32
  long long bidxl = 0;
  float wfloor = 0.f;  // FP64 path: at or below an exact bound a lane of this warp reached
  const F32K<float> K32 = f32_spectral_consts(C);
  for (int r = cta * nwq + wq; r < rows; r += ncta * nwq) {
    const long long o0 = node_index<S>(B, 0, r % ny + 1, r / ny + 1), e0 = (long long)nx * r - 1;
    for (int i = 1 + lane; i <= nx; i += 32) {
      const long long o = o0 + i;
      const S u = q[NP * fs + o], v = q[(NP + 1) * fs + o], w = q[(NP + 2) * fs + o];
      if constexpr (std::is_same<S, float>::value) {
        // the FP32-mixed step sets dt from the FP32 bound f32_spectral_exact
        // (also its initial dt): the argmax of that same value, at every node
        const float sv = f32_spectral_exact(K32, u, v, w);
        if (sv > bestf) {
          bestf = sv;
          bidxl = e0 + i;
        }
      } else {
        if (__fmul_rn(spectral_est_f32(C, u, v, w), 1.00001f) >= wfloor) {
          // exact FP64 bound only where an FP32 estimate (relative error < 1e-6)
          // raised by 1e-5 could reach the running maximum: the argmax is unchanged
          const double sv = spectral_f64(C, u, v, w);
          if (sv > best) {
            best = sv;
            bidx = (double)(e0 + i);
          }
        }
        // a warp-shared floor (a value some lane's node attained exactly), so that
        // the FP64 path runs only when a node of the warp could reach it:
        // non-negative floats order like their bit patterns
        const float bf = best > 0.0 ? __double2float_rd(best) : 0.f;
        wfloor = fmaxf(wfloor, __uint_as_float(__reduce_max_sync(__activemask(), __float_as_uint(bf))));
      }
    }
  }
  if constexpr (std::is_same<S, float>::value) {
    if (bestf >= 0.f) {
      best = (double)bestf;
      bidx = (double)bidxl;
    }
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
    out2[0] = best;
    out2[1] = bidx;
  }
}

// the argmax of the state being reversed, with the FP32 sweep's second level
// of the gather's node sums
template <class S>
__global__ void __launch_bounds__(256) k_adj_argmax(AdjArgs a) {
  adj_argmax_part<S>(a.B, a.C, a.g, blockIdx.x, gridDim.x, a.argpart + 2 * blockIdx.x);
  const int w = threadIdx.x >> 5;
  if (a.ngpart > 0) {
    // second level of the gather's node sums: this CTA's contiguous run of
    // its per-CTA partials, in a fixed order (strided thread sums, a fixed
    // shuffle tree, warps in order)
    const long long lo = (long long)blockIdx.x * a.ngpart / gridDim.x;
    const long long hi = (long long)(blockIdx.x + 1) * a.ngpart / gridDim.x;
    double g3[3] = {0.0, 0.0, 0.0};
    for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x)
      for (int c = 0; c < 3; ++c) g3[c] += a.gpart[3 * q + c];
    __shared__ double sg[8][3];
    for (int c = 0; c < 3; ++c) g3[c] = warp_sum(g3[c]);
    if ((threadIdx.x & 31) == 0)
      for (int c = 0; c < 3; ++c) sg[w][c] = g3[c];
    __syncthreads();
    if (threadIdx.x < 3) {
      double acc = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) acc += sg[q][threadIdx.x];
      a.gpart2[3 * blockIdx.x + threadIdx.x] = acc;
    }
  }
}

// The argmax of every state of a recomputed segment (it depends on the
// forward state only): grid (parts, slots), slot s's state in buffer set 0 of
// blocks[s]; (max, index) pairs at argpart[2 (s parts + part)].
template <class S>
__global__ void __launch_bounds__(256) k_adj_argmax_seg(const BlockDev *blocks, CavConst C, AdjGeom g,
                                                         double *argpart) {
  adj_argmax_part<S>(blocks[blockIdx.y], C, g, blockIdx.x, gridDim.x,
                     argpart + 2 * ((long long)blockIdx.y * gridDim.x + blockIdx.x));
}

// dt = cfl / S: add (-cfl dtbar / S^2) d(bound)/dV at the argmax node.  One
// CTA of kAdjDtThreads: the per-CTA (max, index) pairs of k_adj_argmax are
// reduced in parallel (largest value, smallest index among equals), then one
// thread differentiates the bound at that node (FP64).
constexpr int kAdjDtThreads = 1024;
template <class S, class A>
__global__ void __launch_bounds__(kAdjDtThreads) k_adj_dt(AdjArgs a, int nparts) {
  __shared__ double sb[kAdjDtThreads], si[kAdjDtThreads];
  const int tid = threadIdx.x;
  double best = -1.0, bidx = 0.0;
  for (int q = tid; q < nparts; q += kAdjDtThreads)
    if (a.argpart[2 * q] > best || (a.argpart[2 * q] == best && a.argpart[2 * q + 1] < bidx)) {
      best = a.argpart[2 * q];
      bidx = a.argpart[2 * q + 1];
    }
  sb[tid] = best;
  si[tid] = bidx;
  // the FP32 gather's node sums (dtbar, g sigma bar, floor bar): its per-CTA
  // partials, reduced in a fixed order
  __shared__ double sg[3][kAdjDtThreads];
  double g3[3] = {0.0, 0.0, 0.0};
  // k_adj_argmax's second-level sums, or (gpart2 null) the gather's per-CTA
  // partials themselves
  const double *gp = a.gpart2 ? a.gpart2 : a.gpart;
  const int ng2 = a.ngpart > 0 ? (a.gpart2 ? nparts : a.ngpart) : 0;
  for (int q = tid; q < ng2; q += kAdjDtThreads)
    for (int c = 0; c < 3; ++c) g3[c] += gp[3 * (long long)q + c];
  for (int c = 0; c < 3; ++c) sg[c][tid] = g3[c];
  __syncthreads();
  for (int o = kAdjDtThreads / 2; o > 0; o >>= 1) {
    if (tid < o) {
      if (sb[tid + o] > sb[tid] || (sb[tid + o] == sb[tid] && si[tid + o] < si[tid])) {
        sb[tid] = sb[tid + o];
        si[tid] = si[tid + o];
      }
      for (int c = 0; c < 3; ++c) sg[c][tid] += sg[c][tid + o];
    }
    __syncthreads();
  }
  if (tid != 0) return;
  if (a.ngpart > 0) {
    a.scal[kScDtbar] = sg[0][0];
    a.scal[kScGs] = sg[1][0];
    a.scal[kScFloor] = sg[2][0];
  }
  best = sb[0];
  bidx = si[0];
  const long long e = (long long)bidx;
  int i, j, k;
    unflat(a.g, (unsigned)e, i, j, k);
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
  A *Q = arr<A>(a.Q);
  for (int d = 0; d < 3; ++d)
    Q[aidx(a.g, 1 + d, i, j, k)] += (A)(vbar[d] + (floored ? 0.0 : 2.0 * V[d] * b2bar));
  // the step's Ra adjoint from the buoyancy (g sigma = Ra Pr) and floor
  // (kappa u_ref^2 = kappa Ra Pr) sums; the per-step scalars reset
  a.scal[kScRa] += a.C.nu * a.scal[kScGs] + a.dfloor * a.scal[kScFloor];
  a.scal[kScDtbar] = 0.0;
  a.scal[kScSumP] = 0.0;
  a.scal[kScGs] = 0.0;
  a.scal[kScFloor] = 0.0;
}

// wall and ghost adjoints onto the interior nodes they are formed from
template <class A>
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
  A *Q = arr<A>(a.Q);
  const int ax = face >> 1, high = face & 1;
  const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
  const int c1 = (int)(e % n[a1]) + 1, c2 = (int)(e / n[a1]) + 1;
  const int w = high ? n[ax] + 1 : 0, s = high ? -1 : 1;
  int iw[3], i1[3], i2[3], ig[3];
  iw[ax] = w; i1[ax] = w + s; i2[ax] = w + 2 * s; ig[ax] = w - s;
  iw[a1] = i1[a1] = i2[a1] = ig[a1] = c1;
  iw[a2] = i1[a2] = i2[a2] = ig[a2] = c2;
  const A pw = Q[aidx(a.g, 0, iw[0], iw[1], iw[2])], pg = Q[aidx(a.g, 0, ig[0], ig[1], ig[2])];
  atomicAdd(&Q[aidx(a.g, 0, i1[0], i1[1], i1[2])], (A)2 * pw + (A)3 * pg);
  atomicAdd(&Q[aidx(a.g, 0, i2[0], i2[1], i2[2])], -pw - (A)2 * pg);
  const A tw = Q[aidx(a.g, 4, iw[0], iw[1], iw[2])];
  if (ax == 0) {
    if (!high) a.thetabar[(c1 - 1) + (long long)n[1] * (c2 - 1)] += (double)tw;
  } else {
    atomicAdd(&Q[aidx(a.g, 4, i1[0], i1[1], i1[2])], (A)(4.0 / 3.0) * tw);
    atomicAdd(&Q[aidx(a.g, 4, i2[0], i2[1], i2[2])], (A)(-1.0 / 3.0) * tw);
  }
}

// J accumulation during the forward run: J += Nu_hot of cavity 0
__global__ void k_adj_acc_nusselt(const CavState *cs, double *scal) { scal[kScJ] += cs[0].nu_hot; }

}  // namespace bdc
