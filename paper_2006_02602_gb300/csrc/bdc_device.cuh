// Device-side data structures and kernels of the buoyancy-driven-cavity step
// (Xue & Roy, arXiv 2006.02602).  Shared by the C-ABI translation unit only.
//
// Per step, on the handle's stream (one CUDA graph per buffer parity):
//   k_step      fused residual (Eqs. 1-3) + explicit Euler update of every
//               interior node of every block, FP64 residual sums and the
//               spectral-radius max of the new state as per-CTA partials;
//   k_bc        wall conditions (Section 2) and the hot/cold-wall Nusselt
//               sums; the last CTA to finish reduces the partials in a
//               fixed order: residual norms, next dt, centre pressure,
//               Nusselt numbers, time, step, non-finite flag;
//   k_pack      cut-face ghost data -> contiguous buffers (Section 4.5,
//               Listings 1-2, V3): p at depth 2, u, v, w, T at depth 1;
//   k_unpack    buffers -> the neighbour's ghost layers.
//
// Storage: each block holds two buffer sets (ping-pong); a set is NF
// consecutive padded arrays, x fastest.  Local node (i, j, k), i in
// [-1, n+2], sits at element (XO1 - 1 + i) + pitch (j + 1) + plane (k + 1)
// so that node 1 of every row starts on a 32-byte boundary.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace bdc {

constexpr int kNF = 5;           // p, u, v, w, T
constexpr int kMaxCentre = 8;    // 2^3 centre nodes at most
constexpr int kPartStride = 8;   // doubles per step partial: 5 sums, sr max, pad
constexpr int kBcThreads = 128;  // wall positions per k_bc CTA (one per thread)
constexpr int kFinSlices = 16;   // k_finalize CTAs per cavity at most

struct BlockDev {
  int nx, ny, nz;        // interior nodes of the block
  int ox, oy, oz;        // global node index = o + local index
  int pitch;             // elements per row
  int rows;              // ny + 4
  long long plane;       // pitch * rows
  long long fstride;     // elements per field array
  int wall[6];           // face on a cavity wall (-x, +x, -y, +y, -z, +z)
  int nbr[6];            // neighbour block across a cut face, -1 on walls
  int cav;               // cavity this block belongs to
  int tiles_x, tiles_y, tiles_z;
  int tile_begin;        // first partial slot (k_step tile) of this block
  // z chunking of the step kernels: chunks 0 .. tiles_zc-1 of KC planes cover
  // planes 1 .. zsplit, the other tiles_z - tiles_zc chunks split planes
  // zsplit+1 .. nz into fine chunks (kFineKC planes in the FP64 form,
  // kFineKC32 in the FP32 form, whose KC = zsplit / tiles_zc is set at run
  // time).  Scheduling index c runs over every block's
  // coarse tiles first (coarse_begin + local) and the fine ones last
  // (ncoarse + fine_begin + local): the persistent FP64 grid's counter and
  // the FP32 grids' block order both end on short tiles.  Partial slots stay
  // block-major (tile_begin + local tile index), so a cavity's are contiguous.
  int tiles_zc, zsplit, coarse_begin, fine_begin;
  void *base[2];         // buffer sets (field f at base + f * fstride)
};
constexpr int kFineKC = 2, kFineKC32 = 8;

struct CavConst {
  double h[3], ih[3], ih2[3], ihh[3];
  double nu, alpha, gs, t_inf, b2min, c4, cfl, diffsr, inv_dT;
  double inv_nint, inv_nwall;
  // folded coefficients of the FP64 rates: c4 / (2 h_d) (the dissipation
  // weight of |V_d| + sqrt(V_d^2 + 4 beta^2)), nu / h_d^2, alpha / h_d^2,
  // 2 nu sum 1/h_d^2, 2 alpha sum 1/h_d^2, gs T_inf
  double dsc[3], nuhh[3], alhh[3], nu2s, al2s, gst;
  // FP32 copies (rounded to nearest, as a device conversion would) of the
  // constants the FP32 kernels and estimates use, so that no kernel spends
  // FP64-pipe conversions on them: 1/h, 1/(2h), nu/h^2, alpha/h^2, c4/2, gs,
  // T_inf, beta_min^2, the diffusive spectral term, cfl; 1/h^2, c4, nu, alpha
  float fih[3], fh2[3], fnh[3], fah[3];
  float fc4h, fgs, ftinf, fb2min, fdiffsr, fcfl;
  float fihh[3], fc4, fnu, falpha;
  // the spectral bound at rest, S0 = beta_min (1/h_x + 1/h_y + 1/h_z) + the
  // diffusive term (FP64), and 2 beta_min (FP32): the FP64 step's dt filter
  // works on S - S0
  double s0;
  float f2b0;
  int gaxis;
  int gn[3];
  int ncentre;
  int centre_blk[kMaxCentre];
  long long centre_off[kMaxCentre];  // element offset of the node in its field array
  int tile_begin, tile_end;          // k_step CTAs of this cavity
  int slice_q[kFinSlices + 1];       // k_finalize slice g reduces the step partials slice_q[g] .. slice_q[g+1]-1
  double wscale[2];                  // FP32 step's sums of 3 T_w - 4 T_1 + T_2 -> hot, cold wall fluxes: +-h_x^-1 / (2 dT)
  int bc_begin, bc_end;              // k_bc CTAs of this cavity (all wall faces)
  int bc_xend;                       // the x walls' CTAs (the Nusselt partials) come first: bc_begin .. bc_xend-1
  long long wall_off;                // offset of this cavity's wall temperatures
};

// The grid- and parameter-derived members of CavConst (everything but the
// cavity's tile/wall ranges and centre nodes), from the interior node counts
// and resolved parameters.  One definition for every entry point.
inline void set_cav_physics(CavConst &C, const int gn[3], const cavity_params &p) {
  double sih = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double np1 = (double)gn[d] + 1.0;
    C.gn[d] = gn[d];
    C.h[d] = 1.0 / np1;
    C.ih[d] = np1;
    C.ih2[d] = 0.5 * np1;
    C.ihh[d] = np1 * np1;
    sih += C.ihh[d];
  }
  C.nu = p.Pr;
  C.alpha = 1.0;
  C.gs = p.Ra * p.Pr;
  C.t_inf = p.t_inf;
  C.b2min = p.kappa * p.u_ref * p.u_ref;
  C.c4 = p.c4;
  C.cfl = p.cfl;
  C.diffsr = 2.0 * (C.nu > C.alpha ? C.nu : C.alpha) * sih;
  C.inv_dT = 1.0 / (p.t_hot - p.t_cold);
  C.inv_nint = 1.0 / ((double)gn[0] * gn[1] * gn[2]);
  C.inv_nwall = 1.0 / ((double)gn[1] * gn[2]);
  C.wscale[0] = 0.5 * C.ih[0] * C.inv_dT;
  C.wscale[1] = -0.5 * C.ih[0] * C.inv_dT;
  for (int d = 0; d < 3; ++d) {
    C.dsc[d] = 0.5 * C.c4 * C.ih[d];
    C.nuhh[d] = C.nu * C.ihh[d];
    C.alhh[d] = C.alpha * C.ihh[d];
  }
  C.nu2s = 2.0 * C.nu * sih;
  C.al2s = 2.0 * C.alpha * sih;
  C.gst = C.gs * C.t_inf;
  for (int d = 0; d < 3; ++d) {
    C.fih[d] = (float)C.ih[d];
    C.fh2[d] = (float)C.ih2[d];
    C.fnh[d] = (float)(C.nu * C.ihh[d]);
    C.fah[d] = (float)(C.alpha * C.ihh[d]);
    C.fihh[d] = (float)C.ihh[d];
  }
  C.fc4 = (float)C.c4;
  C.fnu = (float)C.nu;
  C.falpha = (float)C.alpha;
  {
    const double b0 = std::sqrt(C.b2min);
    C.s0 = b0 * (C.ih[0] + C.ih[1] + C.ih[2]) + C.diffsr;
    C.f2b0 = (float)(2.0 * b0);
  }
  C.fc4h = (float)(0.5 * C.c4);
  C.fgs = (float)C.gs;
  C.ftinf = (float)C.t_inf;
  C.fb2min = (float)C.b2min;
  C.fdiffsr = (float)C.diffsr;
  C.fcfl = (float)C.cfl;
  C.gaxis = p.gravity_axis;
}

struct CavState {
  double dt;         // dt of the next step
  double c;          // pending centre-pressure shift of the stored p
  double t;          // simulated time
  long long step;    // steps taken
  double res[5];     // RMS dq/dt of the last step
  double nu_hot, nu_cold;
  int flags;         // bit 0: non-finite residual or spectral radius
  int pad;
};

struct StepRecord {   // one step's record in the host-memory step log (the C ABI's cavity_step_record)
  long long step;
  double t, dt;
  double res[5];
  double nu_hot, nu_cold;
  long long flags;
};

struct WallFace {     // one wall face of one block, processed by k_bc
  int block, face;
  int n1, n2;         // face interior extents (faster, slower face axis)
  int cta_begin;      // first k_bc CTA
  int cav;
};

struct ShellFace {    // the two layers next to one cut face, processed by k_shell_f64
  int block, face;
  int n1, n2;         // face interior extents (faster, slower face axis)
  int cta_begin;
};

struct CutFace {      // one cut face of one block, processed by k_pack / k_unpack
  int src, face, dst;
  int nb, nc;         // face extents (faster, slower face axis)
  int cta_begin;
  long long buf_off;  // element offset into the exchange buffer
};

// ---------------------------------------------------------------------------
// storage traits

template <class S> struct XO;
template <> struct XO<double> { static constexpr int v = 4; };
template <> struct XO<float> { static constexpr int v = 8; };  // node 1 starts a 32-byte sector

template <class S>
__device__ __forceinline__ long long node_index(const BlockDev &B, int i, int j, int k) {
  return (long long)(XO<S>::v - 1 + i) + (long long)B.pitch * (j + 1) + B.plane * (k + 1);
}

// Arrays of one buffer set.  FP64 form: p, u, v, w, T.  FP32-mixed form:
// p_hi, p_lo, u, v, w, T_hi, T_lo (p = p_hi + p_lo and T = T_hi + T_lo,
// unevaluated FP32 pairs: their time-step accumulation is compensated).
// NP = arrays of p; the transported fields u, v, w, T start at array NP.
template <class S> struct Store;
template <> struct Store<double> { static constexpr int NA = 5, NP = 1; };
template <> struct Store<float> { static constexpr int NA = 7, NP = 2; };

template <class S>
__device__ __forceinline__ double load_p(const S *base, long long fs, long long o);
template <>
__device__ __forceinline__ double load_p<double>(const double *base, long long, long long o) { return base[o]; }
template <>
__device__ __forceinline__ double load_p<float>(const float *base, long long fs, long long o) {
  return (double)base[o] + (double)base[fs + o];
}
template <class S>
__device__ __forceinline__ void store_p(S *base, long long fs, long long o, double v);
template <>
__device__ __forceinline__ void store_p<double>(double *base, long long, long long o, double v) { base[o] = v; }
template <>
__device__ __forceinline__ void store_p<float>(float *base, long long fs, long long o, double v) {
  const float hi = (float)v;
  base[o] = hi;
  base[fs + o] = (float)(v - (double)hi);
}

// temperature: array NP + 3 (FP64), or the pair NP + 3 (hi), NP + 4 (lo) (FP32-mixed)
template <class S>
__device__ __forceinline__ double load_T(const S *base, long long fs, long long o) {
  return load_p<S>(base + (Store<S>::NP + 3) * fs, fs, o);
}
template <class S>
__device__ __forceinline__ void store_T(S *base, long long fs, long long o, double v) {
  store_p<S>(base + (Store<S>::NP + 3) * fs, fs, o, v);
}

// ---------------------------------------------------------------------------
// deterministic block reductions (fixed shuffle tree, fixed warp order)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// Square root of a positive, normal, finite FP64 value by Newton's method on
// s^2 - q = 0 with a fixed slope: the seed y ~ 1/sqrt(q) comes from the PTX
// instruction rsqrt.approx.ftz.f64 (measured relative error below 1e-6),
// s_0 = q y, then twice s <- s + (q - s^2) y / 2.  The relative error of s
// after a step is about 1.5 e^2 (e the seed's), so the second step lands below
// the FP64 rounding: the result is within one unit in the last place of the
// correctly rounded root (cavity_check_sqrt measures this against CUDA's sqrt).
// It takes about 30% less FP64-pipe time than the library sqrt on GB300.
// Arguments below the normal range or infinite give NaN (the seed is infinite
// or zero): the rates only take it of V_d^2 + 4 beta^2 >= 4 kappa u_ref^2,
// which the parameter check keeps normal.
__device__ __forceinline__ double sqrt_newton(double q) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(q));
  const double hy = 0.5 * y;
  double s = q * y;
  s = fma(fma(-s, s, q), hy, s);
  return fma(fma(-s, s, q), hy, s);
}

// ---------------------------------------------------------------------------
// Per-node rates, Eqs. 1-3, FP64.  Star values: c, x-, x+, y-, y+, z-, z+.
// Rearranged for few FP64 operations (GB300's FP64 pipe is the bound):
//  - beta^2 eps_d / h_d^4 = c4 lambda_d / h_d, so the continuity rate needs no
//    division, and c4 lambda_d / h_d = (|V_d| + sqrt(V_d^2 + 4 beta^2)) c4/(2 h_d);
//  - the central advection and the diffusion of one transported field share
//    the neighbour weights: -a_d (q_+ - q_-) + k (q_+ + q_- - 2 q_c) / h_d^2
//    = (k/h_d^2 - a_d) q_+ + (k/h_d^2 + a_d) q_- - 2 k q_c / h_d^2, with
//    a_d = V_d / (2 h_d); u, v, w share one set of weights (k = nu), T has its
//    own (k = alpha): seven FMAs per field instead of sixteen operations.

struct NodeF64 {
  double p[13];  // c, x-, x+, y-, y+, z-, z+, x-2, x+2, y-2, y+2, z-2, z+2
  double u[7], v[7], w[7], T[7];
};

__device__ __forceinline__ void rates_f64(const CavConst &C, const NodeF64 &n, double r[5]) {
  const double u0 = n.u[0], v0 = n.v[0], w0 = n.w[0];
  const double b2 = fmax(fma(u0, u0, fma(v0, v0, w0 * w0)), C.b2min);
  const double f4 = 4.0 * b2;
  const double ex = (fabs(u0) + sqrt_newton(fma(u0, u0, f4))) * C.dsc[0];
  const double ey = (fabs(v0) + sqrt_newton(fma(v0, v0, f4))) * C.dsc[1];
  const double ez = (fabs(w0) + sqrt_newton(fma(w0, w0, f4))) * C.dsc[2];
  const double p0 = n.p[0];
  const double d4x = fma(6.0, p0, fma(-4.0, n.p[2] + n.p[1], n.p[8] + n.p[7]));
  const double d4y = fma(6.0, p0, fma(-4.0, n.p[4] + n.p[3], n.p[10] + n.p[9]));
  const double d4z = fma(6.0, p0, fma(-4.0, n.p[6] + n.p[5], n.p[12] + n.p[11]));
  const double diss = fma(ex, d4x, fma(ey, d4y, ez * d4z));
  const double divV = fma(n.u[2] - n.u[1], C.ih2[0], fma(n.v[4] - n.v[3], C.ih2[1], (n.w[6] - n.w[5]) * C.ih2[2]));
  r[0] = fma(-b2, divV, -diss);

  // neighbour weights: m = minus side, p = plus side
  const double nxm = fma(u0, C.ih2[0], C.nuhh[0]), nxp = fma(-u0, C.ih2[0], C.nuhh[0]);
  const double nym = fma(v0, C.ih2[1], C.nuhh[1]), nyp = fma(-v0, C.ih2[1], C.nuhh[1]);
  const double nzm = fma(w0, C.ih2[2], C.nuhh[2]), nzp = fma(-w0, C.ih2[2], C.nuhh[2]);
#define BDC_TRANSPORT(q, xm, xp, ym, yp, zm, zp, centre) \
  fma(xp, q[2], fma(xm, q[1], fma(yp, q[4], fma(ym, q[3], fma(zp, q[6], fma(zm, q[5], centre))))))
  // the buoyancy force (Eq. 2) enters the gravity-axis momentum rate with its centre term
  const double buoy = fma(C.gs, n.T[0], -C.gst);
  const double bv = C.gaxis == 1 ? buoy : 0.0, bw = C.gaxis == 2 ? buoy : 0.0;
  r[1] = fma(-(n.p[2] - n.p[1]), C.ih2[0], BDC_TRANSPORT(n.u, nxm, nxp, nym, nyp, nzm, nzp, -C.nu2s * u0));
  r[2] = fma(-(n.p[4] - n.p[3]), C.ih2[1], BDC_TRANSPORT(n.v, nxm, nxp, nym, nyp, nzm, nzp, fma(-C.nu2s, v0, bv)));
  r[3] = fma(-(n.p[6] - n.p[5]), C.ih2[2], BDC_TRANSPORT(n.w, nxm, nxp, nym, nyp, nzm, nzp, fma(-C.nu2s, w0, bw)));
  const double txm = fma(u0, C.ih2[0], C.alhh[0]), txp = fma(-u0, C.ih2[0], C.alhh[0]);
  const double tym = fma(v0, C.ih2[1], C.alhh[1]), typ = fma(-v0, C.ih2[1], C.alhh[1]);
  const double tzm = fma(w0, C.ih2[2], C.alhh[2]), tzp = fma(-w0, C.ih2[2], C.alhh[2]);
  r[4] = BDC_TRANSPORT(n.T, txm, txp, tym, typ, tzm, tzp, -C.al2s * n.T[0]);
#undef BDC_TRANSPORT
}

// spectral-radius bound of one node's state (the dt denominator); square
// roots within one unit in the last place (sqrt_newton), so dt is the
// correctly rounded formula's to a few ulp
__device__ __forceinline__ double spectral_f64(const CavConst &C, double u, double v, double w) {
  const double b2 = fmax(u * u + v * v + w * w, C.b2min);
  const double f4 = 4.0 * b2;
  const double sx = fabs(u) + sqrt_newton(u * u + f4);
  const double sy = fabs(v) + sqrt_newton(v * v + f4);
  const double sz = fabs(w) + sqrt_newton(w * w + f4);
  return 0.5 * (sx * C.ih[0] + sy * C.ih[1] + sz * C.ih[2]) + C.diffsr;
}

// Rates and explicit update of one node: the new p, u, v, w, T in q (p with
// the pending centre shift taken off), the rates in r.  One function for
// k_step_f64 and k_shell_f64, so a node gives the same bits in either.
__device__ __forceinline__ void update_node_f64(const CavConst &C, const NodeF64 &n, double dt, double cshift,
                                                int local_dt, double q[5], double r[5]) {
  rates_f64(C, n, r);
  const double dtn = local_dt ? C.cfl / spectral_f64(C, n.u[0], n.v[0], n.w[0]) : dt;
  q[0] = (n.p[0] - cshift) + dtn * r[0];
  q[1] = n.u[0] + dtn * r[1];
  q[2] = n.v[0] + dtn * r[2];
  q[3] = n.w[0] + dtn * r[3];
  q[4] = n.T[0] + dtn * r[4];
}

// FP32 estimate of spectral_f64 (the same formula: relative error below
// 1e-6; beta_min^2 = kappa u_ref^2 is at least FP32's smallest normal, so the
// estimate is finite).  The FP64 adjoint's argmax skips a node whose estimate,
// raised by 1e-5, stays below a value the exact FP64 maximum already reached
// (the FP64 step filters on spectral_dev_f32 below instead).
__device__ __forceinline__ float spectral_est_f32(const CavConst &C, float uf, float vf, float wf) {
  const float b2 = fmaxf(__fmaf_rn(uf, uf, __fmaf_rn(vf, vf, __fmul_rn(wf, wf))), C.fb2min);
  const float f4 = __fmul_rn(4.f, b2);
  const float qx = __fmaf_rn(uf, uf, f4), qy = __fmaf_rn(vf, vf, f4), qz = __fmaf_rn(wf, wf, f4);
  float rx, ry, rz;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rx) : "f"(qx));
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ry) : "f"(qy));
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rz) : "f"(qz));
  const float sx = __fmaf_rn(qx, rx, fabsf(uf)), sy = __fmaf_rn(qy, ry, fabsf(vf)), sz = __fmaf_rn(qz, rz, fabsf(wf));
  return __fmaf_rn(0.5f, __fmaf_rn(sx, C.fih[0], __fmaf_rn(sy, C.fih[1], __fmul_rn(sz, C.fih[2]))), C.fdiffsr);
}
// |x| as FP32, rounded toward zero, from the FP64 bit pattern by integer
// operations (a conversion instruction would take slots of GB300's narrow
// FP64 pipe): the exponent rebiased from 1023 to 127, the significand cut to
// 23 bits.  Relative error below 2^-23 in FP32's normal range; exponents
// below it give a value below 2^-125, above it (and inf/NaN) a finite value
// of FP32's largest exponent.
__device__ __forceinline__ float abs_f32_trunc(double x) {
  const unsigned lo = (unsigned)__double2loint(x), hi = (unsigned)__double2hiint(x);
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned m = __funnelshift_l(lo, hi, 3) & 0x7fffffu;  // significand bits 51..29
  const int ec = min(max(e, 896), 1150);
  return __uint_as_float(((unsigned)(ec - 896) << 23) | m);
}
__device__ __forceinline__ float spectral_est_f32(const CavConst &C, double u, double v, double w) {
  return spectral_est_f32(C, abs_f32_trunc(u), abs_f32_trunc(v), abs_f32_trunc(w));
}

// FP32 estimate of D = S - S0, the spectral bound less its value at rest,
// from |u|, |v|, |w| >= 0.  With beta^2 = max(|V|^2, beta_min^2),
// sqrt(V_d^2 + 4 beta^2) - 2 beta_min = (V_d^2 + 4 (beta^2 - beta_min^2)) /
// (sqrt(V_d^2 + 4 beta^2) + 2 beta_min): every term is non-negative, so D
// comes out with a relative error of a few 1e-7 however small it is next to
// S0 (an estimate of S itself has its error on the scale of S0, which near
// rest exceeds the spread of S over the nodes).
__device__ __forceinline__ float spectral_dev_f32(const CavConst &C, float uf, float vf, float wf) {
  const float vv = __fmaf_rn(uf, uf, __fmaf_rn(vf, vf, __fmul_rn(wf, wf)));
  const float f4 = __fmul_rn(4.f, fmaxf(vv, C.fb2min));
  const float d4 = __fmul_rn(4.f, fmaxf(__fsub_rn(vv, C.fb2min), 0.f));  // 4 (beta^2 - beta_min^2)
  const float V[3] = {uf, vf, wf};
  float acc = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float q = __fmaf_rn(V[d], V[d], f4);
    float r, rd;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
    const float den = __fmaf_rn(q, r, C.f2b0);
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd) : "f"(den));
    const float term = __fmaf_rn(__fmaf_rn(V[d], V[d], d4), rd, V[d]);
    acc = __fmaf_rn(term, C.fih[d], acc);
  }
  return __fmul_rn(0.5f, acc);
}

// Order-preserving map of a float (either sign) to a signed int, so that a
// warp can take a float maximum with __reduce_max_sync, and its inverse.
__device__ __forceinline__ int float_key(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float key_float(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// ---------------------------------------------------------------------------
// k_step, FP64: one thread per (i, j) column of a TX x TY tile, sweeping a
// chunk of KC planes in k.  The z-neighbours live in register queues
// (5 deep for p, 3 deep for u, v, w, T); x/y neighbours come through L1.

struct StepArgs {
  const BlockDev *blocks;
  int nblocks;
  const CavConst *cc;
  const CavState *cs;
  double *partials;  // [tile][kPartStride]
  int parity;        // read base[parity], write base[parity ^ 1]
  int mode;          // 0 = step, 1 = spectral radius of the current state only
  unsigned int *sfloor;        // per cavity: the largest published dt-filter floor of this step
                               // (float_key ^ 0x80000000, 0 = none; reset by the next k_bc); null: none
  unsigned int *tile_counter;  // persistent CTAs fetch tiles from it (reset by the next k_bc);
                               // null: one CTA per tile
  int ntiles;
  int local_dt;                // 1: each node at dt_n = cfl / S_n of its state (pseudo time)
  int skip_shell;              // 1: leave the nodes within two layers of a cut face to k_shell_f64
  int ncoarse;                 // coarse tiles of all blocks (scheduling indices below it)
};

// whether local node (i, j, k) of B lies within two layers of one of B's cut
// faces with index below `faces` (all six: faces = 6)
__device__ __forceinline__ bool in_shell(const BlockDev &B, int i, int j, int k, int faces) {
  const int x[3] = {i, j, k}, n[3] = {B.nx, B.ny, B.nz};
  for (int f = 0; f < faces; ++f) {
    if (B.wall[f]) continue;
    const int a = f >> 1;
    if ((f & 1) ? x[a] >= n[a] - 1 : x[a] <= 2) return true;
  }
  return false;
}

__device__ __forceinline__ int find_block(const BlockDev *blocks, int nblocks, int cta) {
  int lo = 0, hi = nblocks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (blocks[mid].tile_begin <= cta) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The tile of scheduling index c: its block, x/y tile, plane range and
// partial slot (coarse chunks of KC planes, fine chunks of KF planes, as
// described at BlockDev).
struct TileRef {
  int b, tx, ty, k0, k1, slot;
};

template <int KC, int KF>
__device__ __forceinline__ TileRef tile_ref(const BlockDev *blocks, int nblocks, int ncoarse, int c) {
  const bool coarse = c < ncoarse;
  const int u = coarse ? c : c - ncoarse;
  // the last block whose first tile of this class is at or before u (blocks
  // without tiles of the class share their successor's start and are passed)
  int lo = 0, hi = nblocks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int begin = coarse ? blocks[mid].coarse_begin : blocks[mid].fine_begin;
    if (begin <= u) lo = mid; else hi = mid - 1;
  }
  const BlockDev &B = blocks[lo];
  const int l = u - (coarse ? B.coarse_begin : B.fine_begin);
  TileRef T;
  T.b = lo;
  T.tx = l % B.tiles_x;
  T.ty = (l / B.tiles_x) % B.tiles_y;
  const int zl = l / (B.tiles_x * B.tiles_y);
  T.k0 = coarse ? zl * KC + 1 : B.zsplit + zl * KF + 1;
  T.k1 = coarse ? min(T.k0 + KC - 1, B.zsplit) : min(T.k0 + KF - 1, B.nz);
  const int tz = coarse ? zl : B.tiles_zc + zl;
  T.slot = B.tile_begin + T.tx + B.tiles_x * (T.ty + B.tiles_y * tz);
  return T;
}

template <int KC>
__device__ __forceinline__ TileRef f64_tile(const StepArgs &a, int c) {
  return tile_ref<KC, kFineKC>(a.blocks, a.nblocks, a.ncoarse, c);
}

// wfloor: a warp-uniform FP32 value of D = S - S0 at or below the one of an
// exact spectral value of this step that some lane of the warp -- or, through
// the cavity's published floor, of any CTA -- has already recorded, lowered
// by 1e-13 of that value (more than the FP64 rounding of S, of S0 and of
// their difference); -inf before the first.  A node whose estimate of D,
// raised by 1e-5 (over 10x its error), stays at or below wfloor cannot raise
// the maximum, so only the others are evaluated in FP64 and the maximum --
// hence dt -- is exactly the FP64 one.  Carried across the warp's tiles of
// one cavity (`fcav`: the cavity it belongs to; a tile of another cavity,
// in a batch, starts again from -inf).
template <int TX, int TY, int KC>
__device__ __forceinline__ void step_tile_f64(const StepArgs &a, int cta, float &wfloor, int &fcav) {
  constexpr int NT = TX * TY;
  const TileRef tile = f64_tile<KC>(a, cta);
  const BlockDev &B = a.blocks[tile.b];
  const CavConst &C = a.cc[B.cav];
  if (B.cav != fcav) {
    wfloor = -INFINITY;
    fcav = B.cav;
  }
  // the cavity's floor as published by every CTA so far this step (a value
  // at or below an exact spectral value some warp recorded): warps far from
  // the maximum start near it too
  if (a.mode == 0 && a.sfloor) {
    const unsigned u = *(volatile const unsigned *)&a.sfloor[B.cav];
    if (u != 0u) wfloor = fmaxf(wfloor, key_float((int)(u ^ 0x80000000u)));
  }
  float published = wfloor;
  const int i = tile.tx * TX + threadIdx.x + 1;
  const int j = tile.ty * TY + threadIdx.y + 1;
  const int k0 = tile.k0;
  const int k1 = tile.k1;
  const bool active = (i <= B.nx) && (j <= B.ny);
  const double dt = a.cs[B.cav].dt;
  const double cshift = a.cs[B.cav].c;

  const double *__restrict__ src = (const double *)B.base[a.parity];
  double *__restrict__ dst = (double *)B.base[a.parity ^ 1];
  const long long fs = B.fstride;
  const double *__restrict__ P = src;
  const double *__restrict__ U = src + fs;
  const double *__restrict__ V = src + 2 * fs;
  const double *__restrict__ W = src + 3 * fs;
  const double *__restrict__ TT = src + 4 * fs;
  const long long pl = B.plane, pt = B.pitch;

  double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, smax = 0;
  if (active) {
    long long o = node_index<double>(B, i, j, k0);
    // z queues: p at k-2..k+1, the others at k-1..k
    double pq0 = __ldg(P + o - 2 * pl), pq1 = __ldg(P + o - pl), pq2 = __ldg(P + o), pq3 = __ldg(P + o + pl);
    double uq0 = __ldg(U + o - pl), uq1 = __ldg(U + o);
    double vq0 = __ldg(V + o - pl), vq1 = __ldg(V + o);
    double wq0 = __ldg(W + o - pl), wq1 = __ldg(W + o);
    double Tq0 = __ldg(TT + o - pl), Tq1 = __ldg(TT + o);
    for (int k = k0; k <= k1; ++k, o += pl) {
      NodeF64 n;
      const double pq4 = __ldg(P + o + 2 * pl);
      const double uq2 = __ldg(U + o + pl), vq2 = __ldg(V + o + pl), wq2 = __ldg(W + o + pl), Tq2 = __ldg(TT + o + pl);
      if (a.mode == 0 && a.skip_shell && in_shell(B, i, j, k, 6)) {
        // computed by k_shell_f64 (interior/shell split)
      } else if (a.mode == 0) {
        n.p[0] = pq2; n.p[5] = pq1; n.p[6] = pq3; n.p[11] = pq0; n.p[12] = pq4;
        n.p[1] = __ldg(P + o - 1); n.p[2] = __ldg(P + o + 1);
        n.p[7] = __ldg(P + o - 2); n.p[8] = __ldg(P + o + 2);
        n.p[3] = __ldg(P + o - pt); n.p[4] = __ldg(P + o + pt);
        n.p[9] = __ldg(P + o - 2 * pt); n.p[10] = __ldg(P + o + 2 * pt);
#define BDC_LOAD7(arr, F, q0, q1, q2)                                           \
  arr[0] = q1; arr[5] = q0; arr[6] = q2;                                        \
  arr[1] = __ldg(F + o - 1); arr[2] = __ldg(F + o + 1);                         \
  arr[3] = __ldg(F + o - pt); arr[4] = __ldg(F + o + pt);
        BDC_LOAD7(n.u, U, uq0, uq1, uq2)
        BDC_LOAD7(n.v, V, vq0, vq1, vq2)
        BDC_LOAD7(n.w, W, wq0, wq1, wq2)
        BDC_LOAD7(n.T, TT, Tq0, Tq1, Tq2)
#undef BDC_LOAD7
        double r[5], qn[5];
        update_node_f64(C, n, dt, cshift, a.local_dt, qn, r);
        const double un = qn[1], vn = qn[2], wn = qn[3];
        for (int f = 0; f < 5; ++f) dst[o + f * fs] = qn[f];
        s0 += r[0] * r[0]; s1 += r[1] * r[1]; s2 += r[2] * r[2]; s3 += r[3] * r[3]; s4 += r[4] * r[4];
        float best = -INFINITY;
        const float dest = spectral_dev_f32(C, abs_f32_trunc(un), abs_f32_trunc(vn), abs_f32_trunc(wn));
        if (__fmul_rn(dest, 1.00001f) > wfloor) {
          const double e = spectral_f64(C, un, vn, wn);
          smax = fmax(smax, e);
          best = __double2float_rd((e - C.s0) - 1e-13 * e);
        }
        // share over the lanes sweeping this tile (all active lanes run the same k range)
        const unsigned am = __activemask();
        wfloor = fmaxf(wfloor, key_float(__reduce_max_sync(am, float_key(best))));
        if (wfloor > published && a.sfloor) {  // publish a rise for the other warps
          if ((int)(threadIdx.x & 31) == __ffs(am) - 1)
            atomicMax(&a.sfloor[B.cav], (unsigned)float_key(wfloor) ^ 0x80000000u);
          published = wfloor;
        }
      } else {
        smax = fmax(smax, spectral_f64(C, uq1, vq1, wq1));
      }
      pq0 = pq1; pq1 = pq2; pq2 = pq3; pq3 = pq4;
      uq0 = uq1; uq1 = uq2; vq0 = vq1; vq1 = vq2; wq0 = wq1; wq1 = wq2; Tq0 = Tq1; Tq1 = Tq2;
    }
  }
  // deterministic CTA reduction of the six partials
  __shared__ double red[NT / 32][6];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2); s3 = warp_sum(s3); s4 = warp_sum(s4);
  smax = warp_max(smax);
  if (lane == 0) {
    red[wid][0] = s0; red[wid][1] = s1; red[wid][2] = s2; red[wid][3] = s3; red[wid][4] = s4; red[wid][5] = smax;
  }
  __syncthreads();
  if (tid < 6) {
    double acc = red[0][tid];
    for (int q = 1; q < NT / 32; ++q) acc = (tid == 5) ? fmax(acc, red[q][tid]) : acc + red[q][tid];
    a.partials[(long long)tile.slot * kPartStride + tid] = acc;
  }
}

// Persistent form: as many CTAs as fit on the GPU at once take tiles in
// order from a counter, so the last round is short (one CTA per tile left a
// partial wave of up to a third of the step on 152 SMs); the counter hands
// out every block's 8-plane tiles before the 2-plane tail tiles.  Partials
// stay indexed by tile slot: the reductions do not depend on which CTA took
// a tile.
template <int TX, int TY, int KC>
__global__ void __launch_bounds__(TX *TY) k_step_f64(StepArgs a) {
  float wfloor = -INFINITY;
  int fcav = -1;
  if (!a.tile_counter) {
    step_tile_f64<TX, TY, KC>(a, blockIdx.x, wfloor, fcav);
    return;
  }
  __shared__ int s_tile;
  const int tid = threadIdx.y * TX + threadIdx.x;
  for (;;) {
    if (tid == 0) s_tile = (int)atomicAdd(a.tile_counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= a.ntiles) break;
    step_tile_f64<TX, TY, KC>(a, tile, wfloor, fcav);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// k_shell_f64: the nodes within two layers of a cut face (the interior/shell
// split of Section 4.7).  They are stepped first, so that the exchange of the
// new ghost layers can run on a second stream while k_step_f64 (skip_shell)
// steps the rest.  One thread per (layer, face position) of each cut face;
// a node near an edge belongs to the first cut face (in face order) within
// two layers of it.  Partials: one slot per CTA after the tiles' slots.

struct ShellArgs {
  const BlockDev *blocks;
  const ShellFace *faces;
  int nfaces;
  const CavConst *cc;
  const CavState *cs;
  double *partials;       // slot part_off + cta
  long long part_off;
  int parity;
  int local_dt;
};

constexpr int kShellThreads = 256;

static __global__ void __launch_bounds__(kShellThreads) k_shell_f64(ShellArgs a) {
  const int cta = blockIdx.x, tid = threadIdx.x;
  int lo = 0, hi = a.nfaces - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.faces[mid].cta_begin <= cta) lo = mid; else hi = mid - 1;
  }
  const ShellFace &F = a.faces[lo];
  const BlockDev &B = a.blocks[F.block];
  const CavConst &C = a.cc[B.cav];
  double s[5] = {0, 0, 0, 0, 0}, smax = 0.0;
  const long long per_layer = (long long)F.n1 * F.n2;
  const long long e = (long long)(cta - F.cta_begin) * kShellThreads + tid;
  if (e < 2 * per_layer) {
    const int d = (int)(e / per_layer) + 1;
    const long long r2 = e % per_layer;
    const int ax = F.face >> 1, hi_face = F.face & 1;
    const int n[3] = {B.nx, B.ny, B.nz};
    int x[3];
    x[ax] = hi_face ? n[ax] + 1 - d : d;
    x[ax == 0 ? 1 : 0] = (int)(r2 % F.n1) + 1;
    x[ax == 2 ? 1 : 2] = (int)(r2 / F.n1) + 1;
    if (!in_shell(B, x[0], x[1], x[2], F.face)) {  // not claimed by an earlier cut face
      const double *src = (const double *)B.base[a.parity];
      double *dst = (double *)B.base[a.parity ^ 1];
      const long long fs = B.fstride, pt = B.pitch, pl = B.plane;
      const long long o = node_index<double>(B, x[0], x[1], x[2]);
      NodeF64 nd;
      const long long po[13] = {0, -1, 1, -pt, pt, -pl, pl, -2, 2, -2 * pt, 2 * pt, -2 * pl, 2 * pl};
      for (int q = 0; q < 13; ++q) nd.p[q] = __ldg(src + o + po[q]);
      for (int q = 0; q < 7; ++q) {
        nd.u[q] = __ldg(src + fs + o + po[q]);
        nd.v[q] = __ldg(src + 2 * fs + o + po[q]);
        nd.w[q] = __ldg(src + 3 * fs + o + po[q]);
        nd.T[q] = __ldg(src + 4 * fs + o + po[q]);
      }
      const CavState &st = a.cs[B.cav];
      double r[5], qn[5];
      update_node_f64(C, nd, st.dt, st.c, a.local_dt, qn, r);
      for (int f = 0; f < 5; ++f) {
        dst[o + f * fs] = qn[f];
        s[f] = r[f] * r[f];
      }
      smax = spectral_f64(C, qn[1], qn[2], qn[3]);
    }
  }
  __shared__ double red[kShellThreads / 32][6];
  const int lane = tid & 31, wid = tid >> 5;
  for (int f = 0; f < 5; ++f) s[f] = warp_sum(s[f]);
  smax = warp_max(smax);
  if (lane == 0) {
    for (int f = 0; f < 5; ++f) red[wid][f] = s[f];
    red[wid][5] = smax;
  }
  __syncthreads();
  if (tid < 6) {
    double acc = red[0][tid];
    for (int q = 1; q < kShellThreads / 32; ++q) acc = (tid == 5) ? fmax(acc, red[q][tid]) : acc + red[q][tid];
    a.partials[(a.part_off + cta) * kPartStride + tid] = acc;
  }
}

// ---------------------------------------------------------------------------
// k_bc (wall conditions + Nusselt partials) and k_finalize (reduction of the
// partials, state advance).

// k_pack / k_unpack / the finalise's exchange CTAs (below)
struct ExchArgs {
  const BlockDev *blocks;
  const CutFace *faces;
  int nfaces;
  double *buf;   // FP64 storage: values; FP32 storage: reinterpreted as float
  int parity;
};

struct BcArgs {
  const BlockDev *blocks;
  const WallFace *faces;
  int nfaces;
  const CavConst *cc;
  CavState *cs;
  int ncav;
  const double *step_partials;
  double *bc_partials;        // [k_bc cta][2]
  unsigned int *counter;      // per cavity: k_finalize slices done
  const double *t_wall;       // hot walls then cold walls, per cavity at wall_off
  unsigned int *tile_counter; // the persistent step kernel's tile counter: reset here
  unsigned int *sfloor;       // the step kernel's per-cavity dt-filter floors: reset here
  long long shell_begin, shell_end;  // k_shell_f64 partial slots of this step (single cavity; empty if equal)
  int parity;                 // buffer set holding the new state
  const CutFace *cuts;        // after a step with cut faces: the exchange of the new state, run by
  int ncuts;                  //   the CTAs after the finalise CTAs (null / 0: none)
  void *xbuf;
  int nslices;                // k_finalize CTAs per cavity (1 .. kFinSlices)
  int wall_ctas;              // after an FP64 step: k_bc's CTAs, run in the finalise launch (0: none)
  StepRecord *log;            // after a step: the step log (host memory), or null
  long long log_cap;          // its records per cavity
  int mode;                   // 0 after a step, 1 after init / set_fields,
                              // 3 walls only (k_bc), no reductions,
                              // 4 after an FP32 step (k_finalize only): Nusselt
                              //   sums in the step partials
};

// x / 3 correctly rounded in three FP64 operations (a rounded reciprocal, then
// one residual correction through fused multiply-adds: Markstein, IBM J. Res.
// Dev. 34 (1990)), where a full division is a long dependent FP64 sequence on
// GB300's narrow FP64 pipe.
__device__ __forceinline__ double div3(double x) {
  constexpr double y = 1.0 / 3.0;
  const double q = x * y;
  return fma(fma(-q, 3.0, x), y, q);
}

// Walls of one face node.  u = v = w = 0 and the isothermal T never change
// between steps: they are written (into both buffer sets) only when `other`
// is given (state refresh); every step rewrites p's wall and ghost values and
// the adiabatic T, and reads T next to the x walls for the Nusselt sums.
template <class S>
__device__ __forceinline__ void apply_wall(const BlockDev &B, const CavConst &C, S *base, int face,
                                           int c1, int c2, const double *t_wall, double &nu_h,
                                           double &nu_c, S *other = nullptr) {
  // wall node: coordinate w on the face axis, c1 on the face's faster axis (y
  // for x faces, else x), c2 on the slower one (z, except y for z faces)
  const int axis = face >> 1, high = face & 1;
  const int na = axis == 0 ? B.nx : (axis == 1 ? B.ny : B.nz);
  const int w = high ? na + 1 : 0;
  const int s = high ? -1 : 1;
  const long long W = node_index<S>(B, axis == 0 ? w : c1, axis == 0 ? c1 : (axis == 1 ? w : c2), axis == 2 ? w : c2);
  const long long step = axis == 0 ? 1 : (axis == 1 ? (long long)B.pitch : B.plane);
  const long long N1 = W + s * step, N2 = W + 2 * s * step, G = W - s * step;
  const long long fs = B.fstride;
  constexpr int NP = Store<S>::NP;
  // every load before the first store (the stores go to the wall and ghost
  // nodes, the loads read interior ones, but the compiler cannot tell)
  const double p1 = load_p<S>(base, fs, N1), p2 = load_p<S>(base, fs, N2);
  const double T1 = load_T<S>(base, fs, N1), T2 = load_T<S>(base, fs, N2);
  double tw = 0.0;
  if (axis == 0) {
    const int J = B.oy + c1, K = B.oz + c2;
    const long long widx = (long long)(J - 1) + (long long)C.gn[1] * (K - 1);
    tw = t_wall[C.wall_off + (high ? (long long)C.gn[1] * C.gn[2] : 0) + widx];
  }
  if (other) {
    base[NP * fs + W] = S(0); base[(NP + 1) * fs + W] = S(0); base[(NP + 2) * fs + W] = S(0);
    other[NP * fs + W] = S(0); other[(NP + 1) * fs + W] = S(0); other[(NP + 2) * fs + W] = S(0);
  }
  const double pw = 2.0 * p1 - p2;
  store_p<S>(base, fs, W, pw);
  store_p<S>(base, fs, G, 2.0 * pw - p1);
  if (axis == 0) {
    if (other) {
      store_T<S>(base, fs, W, tw);
      store_T<S>(other, fs, W, tw);
    }
    const double flux = (3.0 * tw - 4.0 * T1 + T2) * (0.5 * C.ih[0]) * C.inv_dT;
    if (high) nu_c += -flux; else nu_h += flux;
  } else {
    store_T<S>(base, fs, W, div3(4.0 * T1 - T2));
  }
}

// ---------------------------------------------------------------------------
// Finalise: one cavity's per-CTA partials reduced in a fixed order and its
// state advanced (residual RMS, spectral maximum -> next dt, Nusselt numbers,
// time, step count, centre pressure).  GB300's FP64 pipe does about two
// lanes per clock per SM, and one dependent FP64 add costs tens of cycles,
// so the FP64 sums are spread over up to kFinSlices CTAs per cavity
// (BcArgs::nslices, contiguous slices of the partials, about 128 partials a
// slice) and every sum is a shallow fixed tree: within a CTA the eight
// fields are transposed through shared memory and summed by 16 threads each
// (an 8-term tree, then four butterfly levels), and the last CTA of a cavity
// combines the slice totals by the same butterfly.  Nusselt sums: the wall
// kernel's partials (modes 0, 1) or the step partials' slots 6 and 7, sums of
// 3 T_w - 4 T_1 + T_2 (mode 4, FP32 step).  After a step of a decomposed
// cavity, CTAs after the finalise CTAs exchange the new state's cut faces.
constexpr int kFinThreads = 128;

__device__ __forceinline__ double fin_comb(int f, double x, double y) { return f == 5 ? fmax(x, y) : x + y; }

// Field f of the NT values in sv[f * NT ..] summed (f == 5: maximum) by the
// 16 threads t = 16 f .. 16 f + 15 of the CTA: thread s of the group takes
// values s, s + 16, .. s + 112 in a 3-level tree, then a butterfly over the
// group; every thread of the group ends with the same total.
template <int NT>
__device__ __forceinline__ double fin_tree(const double *sv, int f, int s) {
  static_assert(NT == 128, "eight fields x 16 threads, eight values a thread");
  const double *p = sv + f * NT + s;
  const double a0 = fin_comb(f, p[0], p[16]), a1 = fin_comb(f, p[32], p[48]);
  const double a2 = fin_comb(f, p[64], p[80]), a3 = fin_comb(f, p[96], p[112]);
  double v = fin_comb(f, fin_comb(f, a0, a1), fin_comb(f, a2, a3));
#pragma unroll
  for (int o = 1; o < 16; o <<= 1) v = fin_comb(f, v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One slice of a cavity's partials, thread tid's in thread-strided order.
template <int NT>
__device__ __forceinline__ void load_slice(const BcArgs &a, long long q0, long long q1, long long b0, long long b1,
                                           long long s0, long long s1, int tid, double acc[8]) {
  for (int f = 0; f < 8; ++f) acc[f] = 0.0;  // the spectral radius is positive: 0 is its identity too
  long long q = q0 + tid;
  if (q < q1) {  // the first partial is taken as it is, not added to zero
    const double2 *pp = reinterpret_cast<const double2 *>(a.step_partials + q * kPartStride);
    const double2 x0 = pp[0], x1 = pp[1], x2 = pp[2], x3 = pp[3];
    acc[0] = x0.x; acc[1] = x0.y; acc[2] = x1.x; acc[3] = x1.y; acc[4] = x2.x; acc[5] = x2.y;
    if (a.mode == 4) { acc[6] = x3.x; acc[7] = x3.y; }
    q += NT;
  }
  for (; q < q1; q += NT) {
    const double *pp = a.step_partials + q * kPartStride;
    for (int f = 0; f < 5; ++f) acc[f] += pp[f];
    acc[5] = fmax(acc[5], pp[5]);
    if (a.mode == 4) {
      acc[6] += pp[6];
      acc[7] += pp[7];
    }
  }
  for (long long r = s0 + tid; r < s1; r += NT) {  // shell-kernel partials
    const double *pp = a.step_partials + r * kPartStride;
    for (int f = 0; f < 5; ++f) acc[f] += pp[f];
    acc[5] = fmax(acc[5], pp[5]);
  }
  for (long long r = b0 + tid; r < b1; r += NT) {
    acc[6] += a.bc_partials[2 * r];
    acc[7] += a.bc_partials[2 * r + 1];
  }
}

// The CTA tree of the threads' slice sums: field f's total ends in threads
// 16 f .. 16 f + 15.
template <int NT>
__device__ __forceinline__ double tree_slice(const double acc[8], double *sv, int tid) {
#pragma unroll
  for (int f = 0; f < 8; ++f) sv[f * NT + tid] = acc[f];
  __syncthreads();
  return fin_tree<NT>(sv, tid >> 4, tid & 15);
}

template <class S, int NT>
__device__ __forceinline__ void exchange_cta(const ExchArgs &a, int cta);
template <class S>
__device__ __forceinline__ int bc_cta(const BcArgs &a, int cta, bool reduce);

// mid: [ncav][kFinSlices][8] slice totals; a.counter: per cavity, zero between launches
template <class S>
__global__ void __launch_bounds__(kFinThreads) k_finalize(BcArgs a, double *mid) {
  constexpr int NT = kFinThreads;
  __shared__ double sv[8 * NT];
  __shared__ double shm[kFinSlices * 8];
  __shared__ double shc[8];
  __shared__ double sht[8];
  __shared__ double sres[8];  // residual norms, Nusselt numbers, time: the step record's values
  __shared__ double sdt;
  __shared__ long long srec;
  __shared__ bool am_last;
  static_assert(kFinSlices * 8 <= NT && kFinSlices == 16, "one slice total per thread, 16 threads a field");
  // the next step kernel (a programmatic dependent) may start its prologue now;
  // it waits for this grid's completion before it reads the state advanced here
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int nsl = a.nslices, tid = threadIdx.x, f = tid >> 4, s = tid & 15;
  int cav;
  if (blockIdx.x >= a.ncav * nsl) {
    const int c = blockIdx.x - a.ncav * nsl;
    if (c >= a.wall_ctas) {
      // the exchange of the new state's cut faces, beside the reductions
      const ExchArgs x{a.blocks, a.cuts, a.ncuts, (double *)a.xbuf, a.parity};
      exchange_cta<S, kFinThreads>(x, c - a.wall_ctas);
      return;
    }
    // a wall CTA (FP64 step): its walls and Nusselt partial, then it arrives
    // at the cavity's counter like a slice (thread 0 wrote the partial)
    cav = bc_cta<S>(a, c, true);
    if (tid == 0) __threadfence();
  } else {
    cav = blockIdx.x / nsl;
  }
  const CavConst &C = a.cc[cav];
  CavState &st = a.cs[cav];
  const bool slice = blockIdx.x < a.ncav * nsl;
  const int g = blockIdx.x - cav * nsl;
  double acc[8];
  if (slice) {
    // slice bounds: the step partials' from the host's table; the wall and
    // shell partials' (after a state refresh, the overlapped schedule) in
    // 32-bit arithmetic (counts far below 2^27)
    const unsigned nb = (a.mode == 4 || a.wall_ctas) ? 0u : (unsigned)(C.bc_end - C.bc_begin);
    const unsigned ns = (unsigned)(a.shell_end - a.shell_begin);
    load_slice<NT>(a, C.slice_q[g], C.slice_q[g + 1], C.bc_begin + nb * g / nsl, C.bc_begin + nb * (g + 1) / nsl,
                   a.shell_begin + ns * g / nsl, a.shell_begin + ns * (g + 1) / nsl, tid, acc);
  }
  // loads for whichever CTA of the cavity comes last, issued while the
  // partials are in flight and first used after the reductions: the new
  // state's centre pressure (at most 8 nodes, written by the step kernel) and
  // the state it advances (written only by that CTA)
  double cp = 0.0, st_t = 0.0, st_dt = 0.0;
  long long st_step = 0;
  int st_flags = 0;
  if (a.mode != 1 && tid < C.ncentre) {
    const BlockDev &B = a.blocks[C.centre_blk[tid]];
    cp = load_p<S>((const S *)B.base[a.parity], B.fstride, C.centre_off[tid]);
  }
  if (tid == 0 || tid == 3) { st_step = st.step; st_flags = st.flags; }
  if (tid == 2) { st_t = st.t; st_dt = st.dt; }
  if (slice) {
    const double tf = tree_slice<NT>(acc, sv, tid);
    if (nsl == 1 && !a.wall_ctas) {
      // the only CTA of the cavity: its totals go straight to the fold
      if (s == 0) shm[f] = tf;
    } else if (s == 0) {
      mid[((long long)cav * kFinSlices + g) * 8 + f] = tf;
      __threadfence();
    }
  }
  const int nwall = a.wall_ctas ? C.bc_end - C.bc_begin : 0;  // the cavity's wall CTAs in this launch
  if (nsl + nwall > 1) {
    __syncthreads();
    if (tid == 0) am_last = atomicAdd(a.counter + cav, 1u) == (unsigned int)(nsl + nwall) - 1u;
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // the slice totals loaded in parallel
    if (tid < nsl * 8) shm[tid] = mid[(long long)cav * kFinSlices * 8 + tid];
  }
  if (tid < 8) shc[tid] = cp;
  if (nwall) {
    // the wall CTAs' Nusselt partials, thread-strided, into fields 6 and 7 of the tree
    double h = 0.0, c = 0.0;
    for (int q = C.bc_begin + tid; q < C.bc_xend; q += NT) {  // the other walls' partials are zeros
      h += a.bc_partials[2LL * q];
      c += a.bc_partials[2LL * q + 1];
    }
    sv[6 * NT + tid] = h;
    sv[7 * NT + tid] = c;
  }
  __syncthreads();
  // the slice totals of field f combined by its 16 threads (slice s in thread
  // 16 f + s, a butterfly over the first nsl), then the wall partials' tree
  double t = s < nsl ? shm[s * 8 + f] : 0.0;
  for (int o = 1; o < nsl; o <<= 1) t = fin_comb(f, t, __shfl_xor_sync(0xffffffffu, t, o));
  if (nwall && f >= 6) t += fin_tree<NT>(sv, f, s);
  // one thread of each field group finishes its field (the FP64 chains run
  // side by side): residual norms, dt, Nusselt numbers; threads 1 and 2 the
  // centre pressure and the time
  if (s == 0) {
    sht[f] = t;
    if (f < 5 && a.mode != 1) {
      const double r = sqrt(t * C.inv_nint);
      st.res[f] = r;
      sres[f] = r;
    }
    if (f == 5) {
      sdt = C.cfl / t;
      st.dt = sdt;
    }
    if (f >= 6) {
      if (a.mode == 4) t *= C.wscale[f - 6];  // sums of 3 T_w - 4 T_1 + T_2 -> wall fluxes
      const double nu = t * C.inv_nwall;
      sres[f - 1] = nu;  // slots 5, 6 of the record's tail
      if (f == 6) st.nu_hot = nu; else st.nu_cold = nu;
    }
  }
  if (tid == 1 && a.mode != 1) {
    // centre pressure of the new state, lexicographic (k, j, i) order; the
    // count is 1, 2, 4 or 8 (one or two nodes per axis), so the scaling is exact
    double csum = 0.0;
    for (int m = 0; m < C.ncentre; ++m) csum += shc[m];
    st.c = csum * (C.ncentre == 8 ? 0.125 : C.ncentre == 4 ? 0.25 : C.ncentre == 2 ? 0.5 : 1.0);
  }
  if (tid == 2 && a.mode != 1) {  // the time after this step
    st_t += st_dt;
    st.t = st_t;
    sres[7] = st_t;
  }
  if (tid == 3 && a.log && a.mode != 1) srec = (st_step % a.log_cap) * a.ncav + cav;  // this step's log record
  __syncthreads();
  if (tid != 0) return;
  bool bad = !isfinite(sht[5]);
  if (a.mode != 1) {
    for (int q = 0; q < 5; ++q) bad = bad || !isfinite(sht[q]);
    st_step += 1;
    st.step = st_step;
  }
  if (bad) {  // atomic: a timed-out wait of the next step kernel may set bit 1 meanwhile
    st_flags |= 1;
    atomicOr(&st.flags, 1);
  }
  if (a.log && a.mode != 1) {  // this step's record, written to host memory
    StepRecord &r = a.log[srec];
    r.step = st_step;
    r.t = sres[7];
    r.dt = sdt;
    for (int q = 0; q < 5; ++q) r.res[q] = sres[q];
    r.nu_hot = sres[5];
    r.nu_cold = sres[6];
    r.flags = st_flags;
  }
  a.counter[cav] = 0u;
}

// k_bc: wall conditions of every wall face node and the Nusselt partials of
// the x walls, one partial pair per CTA (reduced by k_finalize).
// One CTA of the wall conditions: the wall nodes of kBcThreads positions of
// one face (any block size: each thread takes every blockDim.x-th); with
// `reduce`, the CTA's x-wall Nusselt partial (zeros for other faces).  Returns
// the face's cavity.
template <class S>
__device__ __forceinline__ int bc_cta(const BcArgs &a, int cta, bool reduce) {
  __shared__ double sh[kBcThreads / 32];
  const int tid = threadIdx.x, nwarps = blockDim.x / 32;
  int cav = 0;
  if (cta == 0 && tid == 0 && a.tile_counter) *a.tile_counter = 0u;  // the step kernel has finished
  if (cta == 0 && a.sfloor)
    for (int c = tid; c < a.ncav; c += blockDim.x) a.sfloor[c] = 0u;
  double nu_h = 0.0, nu_c = 0.0;
  bool xwall = false, xhigh = false;
  if (a.nfaces > 0) {
    // the face of this CTA: the last one whose first CTA is not after it (a warp-wide search)
    int fi = 0;
    for (int base = 0; base < a.nfaces; base += 32) {
      const int l = base + (tid & 31);
      const unsigned m = __ballot_sync(0xffffffffu, l < a.nfaces && a.faces[l].cta_begin <= cta);
      if (m) fi = base + 31 - __clz(m);
    }
    const WallFace &F = a.faces[fi];
    cav = F.cav;
    xwall = (F.face >> 1) == 0;
    xhigh = F.face & 1;
    for (int sub = tid; sub < kBcThreads; sub += blockDim.x) {
      const int e = (cta - F.cta_begin) * kBcThreads + sub;
      if (e < F.n1 * F.n2) {
        const BlockDev &B = a.blocks[F.block];
        apply_wall<S>(B, a.cc[F.cav], (S *)B.base[a.parity], F.face, e % F.n1 + 1, e / F.n1 + 1, a.t_wall,
                        nu_h, nu_c, a.mode == 1 ? (S *)B.base[a.parity ^ 1] : nullptr);
      }
    }
  }
  if (!reduce) return cav;  // walls only (a stored state's walls made explicit), no reductions
  if (!xwall) {  // only the x walls carry Nusselt sums (a CTA covers one face)
    if (tid == 0) {
      a.bc_partials[2LL * cta] = 0.0;
      a.bc_partials[2LL * cta + 1] = 0.0;
    }
    return cav;
  }
  // a CTA covers one face: the hot (low x) or the cold (high x) sum, the other is zero
  const double v = warp_sum(xhigh ? nu_c : nu_h);
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    double t = 0;
    for (int q = 0; q < nwarps; ++q) t += sh[q];
    a.bc_partials[2LL * cta] = xhigh ? 0.0 : t;
    a.bc_partials[2LL * cta + 1] = xhigh ? t : 0.0;
  }
  return cav;
}

template <class S>
__global__ void __launch_bounds__(kBcThreads) k_bc(BcArgs a) {
  bc_cta<S>(a, blockIdx.x, a.mode != 3);
}

// ---------------------------------------------------------------------------
// k_pack / k_unpack (Section 4.5, Listings 1-2, Optimized V3).  One thread per
// (ib, ic) face position; buffer layout p[(ic nb + ib) 2 + d], then
// var[2 nb nc + v nb nc + ic nb + ib].  Depth d counts layers in increasing
// index order.  Pure copies: bit exact.

__device__ __forceinline__ int find_cut(const CutFace *faces, int nfaces, int cta) {
  int lo = 0, hi = nfaces - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (faces[mid].cta_begin <= cta) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class S>
__device__ __forceinline__ void face_geometry(const BlockDev &B, int face, int ib, int ic, bool ghost,
                                              long long &p_first, long long &v_node, long long &dstep) {
  // face axis a; the face's faster axis (y for x faces, else x) gets ib + 1,
  // the slower one (z, except y for z faces) ic + 1 (selects rather than an
  // indexed array, which would live in local memory)
  const int a = face >> 1, high = face & 1;
  const int na = a == 0 ? B.nx : (a == 1 ? B.ny : B.nz);
  const int b1 = ib + 1, c1 = ic + 1;
  int pl, vl;
  if (!ghost) { pl = high ? na - 1 : 1; vl = high ? na : 1; }
  else { pl = high ? na + 1 : -1; vl = high ? na + 1 : 0; }
  p_first = node_index<S>(B, a == 0 ? pl : b1, a == 0 ? b1 : (a == 1 ? pl : c1), a == 2 ? pl : c1);
  v_node = node_index<S>(B, a == 0 ? vl : b1, a == 0 ? b1 : (a == 1 ? vl : c1), a == 2 ? vl : c1);
  dstep = a == 0 ? 1 : (a == 1 ? (long long)B.pitch : B.plane);
}

template <class S>
__global__ void __launch_bounds__(256) k_pack(ExchArgs a) {
  const int fi = find_cut(a.faces, a.nfaces, blockIdx.x);
  const CutFace &F = a.faces[fi];
  const int e = (blockIdx.x - F.cta_begin) * 256 + threadIdx.x;
  const int plane = F.nb * F.nc;
  if (e >= plane) return;
  const int ib = e % F.nb, ic = e / F.nb;
  const BlockDev &B = a.blocks[F.src];
  const S *q = (const S *)B.base[a.parity];
  long long p_first, v_node, dstep;
  face_geometry<S>(B, F.face, ib, ic, false, p_first, v_node, dstep);
  S *buf = (S *)a.buf + F.buf_off;
  constexpr int NP = Store<S>::NP;  // pressure arrays (FP32-mixed: hi, then lo section)
  for (int pa = 0; pa < NP; ++pa) {
    const S *pq = q + (long long)pa * B.fstride;
    buf[2LL * pa * plane + 2LL * e] = pq[p_first];
    buf[2LL * pa * plane + 2LL * e + 1] = pq[p_first + dstep];
  }
  for (int v = 0; v < Store<S>::NA - NP; ++v)  // u, v, w, T (FP32-mixed: T_hi, T_lo)
    buf[2LL * NP * plane + (long long)v * plane + e] = q[(long long)(NP + v) * B.fstride + v_node];
}

template <class S>
__global__ void __launch_bounds__(256) k_unpack(ExchArgs a) {
  const int fi = find_cut(a.faces, a.nfaces, blockIdx.x);
  const CutFace &F = a.faces[fi];
  const int e = (blockIdx.x - F.cta_begin) * 256 + threadIdx.x;
  const int plane = F.nb * F.nc;
  if (e >= plane) return;
  const int ib = e % F.nb, ic = e / F.nb;
  const BlockDev &B = a.blocks[F.dst];
  S *q = (S *)B.base[a.parity];
  long long p_first, v_node, dstep;
  face_geometry<S>(B, F.face ^ 1, ib, ic, true, p_first, v_node, dstep);
  const S *buf = (const S *)a.buf + F.buf_off;
  constexpr int NP = Store<S>::NP;
  for (int pa = 0; pa < NP; ++pa) {
    S *pq = q + (long long)pa * B.fstride;
    pq[p_first] = buf[2LL * pa * plane + 2LL * e];
    pq[p_first + dstep] = buf[2LL * pa * plane + 2LL * e + 1];
  }
  for (int v = 0; v < Store<S>::NA - NP; ++v)
    q[(long long)(NP + v) * B.fstride + v_node] = buf[2LL * NP * plane + (long long)v * plane + e];
}

// The step's exchange, one CTA of NT threads per 256 face positions
// (CutFace::cta_begin counts such CTAs): the ghost values k_pack followed by
// k_unpack would write, copied straight from the sending block's layers (the
// face buffer is packed only when asked for, by cavity_get_face_buffer).  Run
// by the finalise kernel's extra CTAs beside its reductions, so it is written
// for latency: the face found by a warp-wide search, every value of the
// thread's positions loaded before the first store.
template <class S, int NT>
__device__ __forceinline__ void exchange_cta(const ExchArgs &a, int cta) {
  static_assert(256 % NT == 0, "positions per thread");
  constexpr int NPOS = 256 / NT, NP = Store<S>::NP, NA = Store<S>::NA, NV = NP + NA;  // p at depth 2
  // the face of this CTA: the last one whose first CTA is not after it
  int fi = 0;
  for (int base = 0; base < a.nfaces; base += 32) {
    const int l = base + (threadIdx.x & 31);
    const unsigned m = __ballot_sync(0xffffffffu, l < a.nfaces && a.faces[l].cta_begin <= cta);
    if (m) fi = base + 31 - __clz(m);
  }
  const CutFace F = a.faces[fi];
  const BlockDev &B = a.blocks[F.src];
  const BlockDev &D = a.blocks[F.dst];
  const int plane = F.nb * F.nc;
  const S *__restrict__ q = (const S *)B.base[a.parity];
  S *__restrict__ g = (S *)D.base[a.parity];
  const long long fs = B.fstride, fd = D.fstride;
  int e[NPOS];
  long long gp[NPOS], gv[NPOS], gstep = 0;
  S x[NPOS][NV];
#pragma unroll
  for (int r = 0; r < NPOS; ++r) {
    e[r] = (cta - F.cta_begin) * 256 + r * NT + (int)threadIdx.x;
    if (e[r] >= plane) continue;
    const int ib = e[r] % F.nb, ic = e[r] / F.nb;
    long long p_first, v_node, dstep;
    face_geometry<S>(B, F.face, ib, ic, false, p_first, v_node, dstep);
    face_geometry<S>(D, F.face ^ 1, ib, ic, true, gp[r], gv[r], gstep);
#pragma unroll
    for (int pa = 0; pa < NP; ++pa) {
      x[r][2 * pa] = q[pa * fs + p_first];
      x[r][2 * pa + 1] = q[pa * fs + p_first + dstep];
    }
#pragma unroll
    for (int v = 0; v < NA - NP; ++v) x[r][2 * NP + v] = q[(NP + v) * fs + v_node];
  }
#pragma unroll
  for (int r = 0; r < NPOS; ++r) {
    if (e[r] >= plane) continue;
#pragma unroll
    for (int pa = 0; pa < NP; ++pa) {
      g[pa * fd + gp[r]] = x[r][2 * pa];
      g[pa * fd + gp[r] + gstep] = x[r][2 * pa + 1];
    }
#pragma unroll
    for (int v = 0; v < NA - NP; ++v) g[(NP + v) * fd + gv[r]] = x[r][2 * NP + v];
  }
}

// ---------------------------------------------------------------------------
// initial state, gather / scatter of the interior

// splitmix64 (Steele, Lea & Flood 2014): finaliser of state x + golden gamma
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

struct InitArgs {
  const BlockDev *blocks;
  const CavConst *cc;
  int block;
  int parity;
  unsigned long long seed;
  double noise;
  double t_hot, t_cold;
};

template <class S>
__global__ void k_init(InitArgs a) {
  const BlockDev &B = a.blocks[a.block];
  const long long n = (long long)B.nx * B.ny * B.nz;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int i = (int)(e % B.nx) + 1, j = (int)((e / B.nx) % B.ny) + 1, k = (int)(e / ((long long)B.nx * B.ny)) + 1;
  const CavConst &C = a.cc[B.cav];
  const int I = B.ox + i, J = B.oy + j, K = B.oz + k;
  const uint64_t gidx = (uint64_t)(I - 1) + (uint64_t)C.gn[0] * ((uint64_t)(J - 1) + (uint64_t)C.gn[1] * (uint64_t)(K - 1));
  const double U = (double)(splitmix64(a.seed * (1ULL << 40) + gidx) >> 11) * (1.0 / 9007199254740992.0);
  // explicit round-to-nearest operations (no contraction): the initial state is
  // reproducible bit for bit by any IEEE implementation of the same formula
  const double x = __dmul_rn((double)I, C.h[0]);
  const double lin = __dadd_rn(a.t_hot, __dmul_rn(__dsub_rn(a.t_cold, a.t_hot), x));
  const double pert = __dmul_rn(a.noise, __dsub_rn(__dmul_rn(2.0, U), 1.0));
  store_T<S>((S *)B.base[a.parity], B.fstride, node_index<S>(B, i, j, k), __dadd_rn(lin, pert));
}

// field f (0 = p, 1..4 = u, v, w, T) of node offset o, widened to FP64
template <class S>
__device__ __forceinline__ double get_field(const S *q, long long fs, int f, long long o) {
  if (f == 0) return load_p<S>(q, fs, o);
  if (f == 4) return load_T<S>(q, fs, o);
  return (double)q[(long long)(Store<S>::NP + f - 1) * fs + o];
}
template <class S>
__device__ __forceinline__ void put_field(S *q, long long fs, int f, long long o, double v) {
  if (f == 0) store_p<S>(q, fs, o, v);
  else if (f == 4) store_T<S>(q, fs, o, v);
  else q[(long long)(Store<S>::NP + f - 1) * fs + o] = (S)v;
}

struct MoveArgs {
  const BlockDev *blocks;
  int block;
  int parity;
  int mask;
  int gn[3];
  double *stage;       // [nf][gnz][gny][gnx] FP64, fields of the mask in order
  double pshift;       // subtracted from p on gather
};

template <class S>
__global__ void k_gather(MoveArgs a) {
  const BlockDev &B = a.blocks[a.block];
  const long long n = (long long)B.nx * B.ny * B.nz;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int i = (int)(e % B.nx) + 1, j = (int)((e / B.nx) % B.ny) + 1, k = (int)(e / ((long long)B.nx * B.ny)) + 1;
  const long long g = (long long)(B.ox + i - 1) + (long long)a.gn[0] * ((B.oy + j - 1) + (long long)a.gn[1] * (B.oz + k - 1));
  const long long gN = (long long)a.gn[0] * a.gn[1] * a.gn[2];
  const S *q = (const S *)B.base[a.parity];
  const long long o = node_index<S>(B, i, j, k);
  int slot = 0;
  for (int f = 0; f < kNF; ++f) {
    if (!(a.mask & (1 << f))) continue;
    double v = get_field<S>(q, B.fstride, f, o);
    if (f == 0) v -= a.pshift;
    a.stage[slot * gN + g] = v;
    ++slot;
  }
}

struct BoxArgs {
  const BlockDev *blocks;
  int nblocks;
  int parity;
  int mask;
  int i0, j0, k0, ni, nj, nk;  // global 1-based node box
  double *stage;               // [nf][nk][nj][ni]
  double pshift;
};

template <class S>
__global__ void k_gather_box(BoxArgs a) {
  const long long n = (long long)a.ni * a.nj * a.nk;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int I = a.i0 + (int)(e % a.ni), J = a.j0 + (int)((e / a.ni) % a.nj), K = a.k0 + (int)(e / ((long long)a.ni * a.nj));
  for (int b = 0; b < a.nblocks; ++b) {
    const BlockDev &B = a.blocks[b];
    if (I <= B.ox || I > B.ox + B.nx || J <= B.oy || J > B.oy + B.ny || K <= B.oz || K > B.oz + B.nz) continue;
    const S *q = (const S *)B.base[a.parity];
    const long long o = node_index<S>(B, I - B.ox, J - B.oy, K - B.oz);
    int slot = 0;
    for (int f = 0; f < kNF; ++f) {
      if (!(a.mask & (1 << f))) continue;
      double v = get_field<S>(q, B.fstride, f, o);
      if (f == 0) v -= a.pshift;
      a.stage[slot * n + e] = v;
      ++slot;
    }
    return;
  }
}

template <class S>
__global__ void k_scatter(MoveArgs a) {
  const BlockDev &B = a.blocks[a.block];
  const long long n = (long long)B.nx * B.ny * B.nz;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int i = (int)(e % B.nx) + 1, j = (int)((e / B.nx) % B.ny) + 1, k = (int)(e / ((long long)B.nx * B.ny)) + 1;
  const long long g = (long long)(B.ox + i - 1) + (long long)a.gn[0] * ((B.oy + j - 1) + (long long)a.gn[1] * (B.oz + k - 1));
  const long long gN = (long long)a.gn[0] * a.gn[1] * a.gn[2];
  S *q = (S *)B.base[a.parity];
  const long long o = node_index<S>(B, i, j, k);
  int slot = 0;
  for (int f = 0; f < kNF; ++f) {
    if (!(a.mask & (1 << f))) continue;
    put_field<S>(q, B.fstride, f, o, a.stage[slot * gN + g]);
    ++slot;
  }
}

// p of the stored state is p_true + c: fold a pending shift into the array
// (used before overwriting other fields from the host, so that c can be reset)
template <class S>
__global__ void k_shift_p(const BlockDev *blocks, int block, int parity, double c) {
  const BlockDev &B = blocks[block];
  const long long n = (long long)(B.nx + 4) * (B.ny + 4) * (B.nz + 4);
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int i = (int)(e % (B.nx + 4)) - 1, j = (int)((e / (B.nx + 4)) % (B.ny + 4)) - 1;
  const int k = (int)(e / ((long long)(B.nx + 4) * (B.ny + 4))) - 1;
  S *q = (S *)B.base[parity];
  const long long o = node_index<S>(B, i, j, k);
  store_p<S>(q, B.fstride, o, load_p<S>(q, B.fstride, o) - c);
}

// copy of one stored array of a block (walls and ghosts included) to a dense
// stage; `field` is the array index (FP32-mixed: 0 = p_hi, 1 = p_lo, 2.. = u..T)
template <class S>
__global__ void k_copy_block(const BlockDev *blocks, int block, int parity, int field, double *stage) {
  const BlockDev &B = blocks[block];
  const long long n = (long long)(B.nx + 4) * (B.ny + 4) * (B.nz + 4);
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int i = (int)(e % (B.nx + 4)) - 1, j = (int)((e / (B.nx + 4)) % (B.ny + 4)) - 1;
  const int k = (int)(e / ((long long)(B.nx + 4) * (B.ny + 4))) - 1;
  const S *q = (const S *)B.base[parity];
  stage[e] = (double)q[field * B.fstride + node_index<S>(B, i, j, k)];
}

}  // namespace bdc
