// FP32-mixed form of the fused step (Eqs. 1-3, Section 3.1 stencils): u, v,
// w stored and updated in FP32; p and T stored as unevaluated FP32 pairs
// (hi + lo) and accumulated with an error-free transformation, so their
// time-step accumulation keeps about 48 significant bits (T's rounding would
// otherwise reach w through the buoyancy coefficient Ra Pr); every
// difference of the stencils is formed relative to the centre node (exact in
// FP32 for neighbouring values), hi-minus-hi plus lo-minus-lo for p, so no
// cancellation is lost.  Residual sums are FP32 within a thread's z-chunk and
// a warp's shuffle tree and FP64 from there on; the spectral maximum is FP32.
//
// Wall conditions (Section 2) are applied where the values are read: p's wall
// and ghost values and the adiabatic T are formed from the two interior
// layers next to each wall (the same FP64 formulas as the wall kernel) as
// planes arrive in shared memory (x and y walls) or enter the z queues (z
// walls).  u = v = w = 0 and the isothermal T never change and stay stored.
//
// Data movement (GB300): per CTA a 32 x 8 tile in (x, y) sweeps a KC-plane
// chunk in z.  One elected thread streams whole planes of the tile plus a
// two-node halo with TMA (cp.async.bulk.tensor.4d over x, y, z and the array
// index: all six arrays in one copy) into a ring of R shared-memory slots,
// each guarded by an mbarrier with a bounded wait; the z-neighbours live in
// register queues (5 deep for p, 3 for u, v, w, T).  HBM sees each of the
// seven arrays read once and written once per step: 56 bytes per interior
// point.
#pragma once

#include <cuda.h>

#include "bdc_device.cuh"

namespace bdc {

constexpr int kF32TX = 32, kF32TY = 8, kF32KC = 64, kF32R = 8;  // default tile height, z chunk, ring depth
constexpr int kF32BX = kF32TX + 8;  // x halo 4 on each side: the box starts on a 16-byte boundary
constexpr int kF32NA = 7;           // p_hi, p_lo, u, v, w, T_hi, T_lo
__host__ __device__ constexpr int f32_box_y(int TY) { return TY + 4; }  // y halo 2 (pressure star)
__host__ __device__ constexpr int f32_slot_floats(int TY) { return kF32NA * f32_box_y(TY) * kF32BX; }
__host__ __device__ constexpr int f32_smem_bytes(int TY, int R) { return R * f32_slot_floats(TY) * 4 + R * 8; }
constexpr long long kWaitCycles = 4000000000LL;  // bounded mbarrier wait, about 2 s

struct StepF32Args {
  const BlockDev *blocks;
  int nblocks;
  const CavConst *cc;
  CavState *cs;               // dt and c read; flags bit 1 set on a timed-out wait
  const CUtensorMap *maps;    // [2 * block + parity], in global memory
  double *partials;           // [cta][kPartStride]
  int parity;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase with the given parity, giving up after kWaitCycles
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

// hi/lo difference (a - c) of two FP32 pairs
__device__ __forceinline__ float pdiff(float ah, float al, float ch, float cl) { return (ah - ch) + (al - cl); }

// square root of a positive FP32 value as x * rsqrt(x) (two instructions,
// within a few ulp); the FP32 form uses it for the wave speeds only
__device__ __forceinline__ float sqrt_pos(float x) { return x * rsqrtf(x); }

__device__ __forceinline__ void split2(double v, float &hi, float &lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// a + (a - b) for FP32 pairs: the linear extrapolation 2a - b with the hi
// parts' rounding error carried into lo (two-sum), so about 48 bits survive
__device__ __forceinline__ void extrapolate_pair(float ah, float al, float bh, float bl, float &rh, float &rl) {
  const float d = ah - bh;  // exact for neighbouring values
  const float s = ah + d;
  const float bp = s - ah;
  const float e = (ah - (s - bp)) + (d - bp);
  rh = s;
  rl = e + (al + (al - bl));
}

// wall and ghost pressure from the two layers next to a wall (p1 nearest):
// p_w = 2 p1 - p2, p_g = 2 p_w - p1 (one-sided second-order extrapolation)
__device__ __forceinline__ void wall_pressure(float h1, float l1, float h2, float l2, float &hw, float &lw,
                                              float &hg, float &lg) {
  extrapolate_pair(h1, l1, h2, l2, hw, lw);
  extrapolate_pair(hw, lw, h1, l1, hg, lg);
}

// (h, l) + d for an FP32 pair: two-sum of the hi part, error carried into lo
__device__ __forceinline__ void pair_add(float h, float l, float d, float &rh, float &rl) {
  const float s = h + d;
  const float bp = s - h;
  const float e = (h - (s - bp)) + (d - bp);
  const float lo = l + e;
  rh = s + lo;
  rl = lo - (rh - s);
}

// adiabatic wall temperature (4 T1 - T2) / 3 = T1 + (T1 - T2) / 3 of FP32 pairs
__device__ __forceinline__ void wall_temperature(float h1, float l1, float h2, float l2, float &hw, float &lw) {
  const float d = (h1 - h2) + (l1 - l2);
  pair_add(h1, l1, d * (1.f / 3.f), hw, lw);
}

// Apply the x and y wall conditions to one freshly loaded plane slot.
// Slot coordinates: lx = i - i0 + 4, ly = j - j0 + 2.  Threads [0, BX) take
// the low y wall, [BX, 2BX) the high y wall, the next BY the low x wall and
// the next BY the high x wall (x walls: pressure only; their temperature is
// prescribed and stored).
template <int NT, int BY>
__device__ __forceinline__ void fix_plane_walls(float *s, int tid, bool wxl, bool wxh, bool wyl, bool wyh,
                                                int lxh, int lyh) {
  constexpr int BX = kF32BX, AS = BX * BY;
  float *H = s, *L = s + AS, *TH = s + 5 * AS, *TL = s + 6 * AS;
  static_assert(NT >= 2 * (BX + BY), "thread groups");
  if (wyl && tid < BX) {
    const int x = tid;
    float hw, lw, hg, lg;
    wall_pressure(H[2 * BX + x], L[2 * BX + x], H[3 * BX + x], L[3 * BX + x], hw, lw, hg, lg);
    H[BX + x] = hw; L[BX + x] = lw; H[x] = hg; L[x] = lg;
    wall_temperature(TH[2 * BX + x], TL[2 * BX + x], TH[3 * BX + x], TL[3 * BX + x], TH[BX + x], TL[BX + x]);
  } else if (wyh && tid >= BX && tid < 2 * BX) {
    const int x = tid - BX;
    const int r1 = lyh, r2 = lyh - 1;  // rows of nodes ny and ny - 1
    float hw, lw, hg, lg;
    wall_pressure(H[r1 * BX + x], L[r1 * BX + x], H[r2 * BX + x], L[r2 * BX + x], hw, lw, hg, lg);
    H[(r1 + 1) * BX + x] = hw; L[(r1 + 1) * BX + x] = lw;
    if (r1 + 2 < BY) { H[(r1 + 2) * BX + x] = hg; L[(r1 + 2) * BX + x] = lg; }
    wall_temperature(TH[r1 * BX + x], TL[r1 * BX + x], TH[r2 * BX + x], TL[r2 * BX + x], TH[(r1 + 1) * BX + x],
                     TL[(r1 + 1) * BX + x]);
  } else if (wxl && tid >= 2 * BX && tid < 2 * BX + BY) {
    const int y = tid - 2 * BX;
    float hw, lw, hg, lg;
    wall_pressure(H[y * BX + 4], L[y * BX + 4], H[y * BX + 5], L[y * BX + 5], hw, lw, hg, lg);
    H[y * BX + 3] = hw; L[y * BX + 3] = lw; H[y * BX + 2] = hg; L[y * BX + 2] = lg;
  } else if (wxh && tid >= 2 * BX + BY && tid < 2 * (BX + BY)) {
    const int y = tid - 2 * BX - BY;
    const int c1 = lxh, c2 = lxh - 1;  // columns of nodes nx and nx - 1
    float hw, lw, hg, lg;
    wall_pressure(H[y * BX + c1], L[y * BX + c1], H[y * BX + c2], L[y * BX + c2], hw, lw, hg, lg);
    H[y * BX + c1 + 1] = hw; L[y * BX + c1 + 1] = lw;
    if (c1 + 2 < BX) { H[y * BX + c1 + 2] = hg; L[y * BX + c1 + 2] = lg; }
  }
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <int TY, int KC, int R>
__global__ void __launch_bounds__(kF32TX *TY, 512 / (kF32TX * TY)) k_step_f32(StepF32Args a) {
  static_assert(R >= 4 && (R & (R - 1)) == 0, "ring depth: a power of two >= 4");
  constexpr int TX = kF32TX, NT = TX * TY;
  constexpr int BX = kF32BX, BY = f32_box_y(TY), AS = BX * BY;  // array stride inside a slot
  constexpr int SF = f32_slot_floats(TY), SB = SF * 4;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float *ring = reinterpret_cast<float *>(smem_raw);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + R * SB);

  const int cta = blockIdx.x;
  const int b = find_block(a.blocks, a.nblocks, cta);
  const BlockDev &B = a.blocks[b];
  const CavConst &C = a.cc[B.cav];
  const int t = cta - B.tile_begin;
  const int tx = t % B.tiles_x, ty = (t / B.tiles_x) % B.tiles_y, tz = t / (B.tiles_x * B.tiles_y);
  const int i0 = tx * TX + 1, j0 = ty * TY + 1, k0 = tz * KC + 1;
  const int k1 = min(k0 + KC - 1, B.nz);
  const int li = threadIdx.x, lj = threadIdx.y, tid = lj * TX + li;
  const int i = i0 + li, j = j0 + lj;
  const bool active = (i <= B.nx) && (j <= B.ny);
  const CUtensorMap *map = a.maps + 2 * b + a.parity;
  const int nplanes = (k1 - k0 + 1) + 4;  // z = k0-2 .. k1+2
  const int x0 = XO<float>::v - 1 + i0 - 4, y0 = (j0 - 2) + 1, zbase = (k0 - 2) + 1;
  // walls whose wall/ghost nodes fall inside this tile's boxes
  const bool wxl = B.wall[0] && tx == 0;
  const bool wxh = B.wall[1] && B.nx + 1 <= i0 + TX + 3;
  const bool wyl = B.wall[2] && ty == 0;
  const bool wyh = B.wall[3] && B.ny + 1 <= j0 + TY + 1;
  const bool wzl = B.wall[4], wzh = B.wall[5];
  const bool fix = wxl || wxh || wyl || wyh;
  const int lxh = B.nx - i0 + 4, lyh = B.ny - j0 + 2;

  if (tid == 0) {
    for (int s = 0; s < R; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
  }
  __syncthreads();
  int issued = 0;
  auto issue = [&](int pl) {
    const int s = pl & (R - 1);
    mbar_expect_tx(&bars[s], SB);
    tma_load_4d(ring + s * SF, map, &bars[s], x0, y0, zbase + pl, 0);
  };
  if (tid == 0) {
    for (; issued < min(R, nplanes); ++issued) issue(issued);
  }
  auto wait_plane = [&](int pl) { return mbar_wait_bounded(&bars[pl & (R - 1)], (uint32_t)((pl / R) & 1)); };
  auto slot = [&](int pl) { return ring + (pl & (R - 1)) * SF; };
  const int col = (lj + 2) * BX + (li + 4);  // own column inside a slot

  // constants in FP32
  const float ihx = (float)C.ih[0], ihy = (float)C.ih[1], ihz = (float)C.ih[2];
  const float h2x = (float)C.ih2[0], h2y = (float)C.ih2[1], h2z = (float)C.ih2[2];
  const float nu = (float)C.nu, gs = (float)C.gs, tinf = (float)C.t_inf, b2min = (float)C.b2min;
  const float nhx = (float)(C.nu * C.ihh[0]), nhy = (float)(C.nu * C.ihh[1]), nhz = (float)(C.nu * C.ihh[2]);
  const float ahx = (float)(C.alpha * C.ihh[0]), ahy = (float)(C.alpha * C.ihh[1]), ahz = (float)(C.alpha * C.ihh[2]);
  const float c4h = (float)(0.5 * C.c4), diffsr = (float)C.diffsr;
  const float gy_on = C.gaxis == 1 ? 1.f : 0.f, gz_on = C.gaxis == 2 ? 1.f : 0.f;
  const float dt = (float)a.cs[B.cav].dt;
  const float cshift = (float)a.cs[B.cav].c;
  (void)nu;

  const long long fs = B.fstride;
  // output pointer of this thread's node at plane k0 (advanced one plane per k)
  float *__restrict__ out = (float *)B.base[a.parity ^ 1] + node_index<float>(B, min(i, B.nx), min(j, B.ny), k0);

  bool bad = false;
  // prologue: planes k0-2 .. k0+1 give the initial z queues
  float ph[5], pq[5], uq[3], vq[3], wq[3], Tq[3], Tl[3];
  float T2next = 0.f, T2next_lo = 0.f;  // T at plane k0+1 (z-wall temperature of the bottom chunk)
  for (int pl = 0; pl < 4; ++pl) {
    if (!bad && !wait_plane(pl)) bad = true;
    if (!bad) {
      float *s = slot(pl);
      ph[pl] = s[col];
      pq[pl] = s[AS + col];
      if (pl >= 1 && pl <= 2) {
        uq[pl - 1] = s[2 * AS + col];
        vq[pl - 1] = s[3 * AS + col];
        wq[pl - 1] = s[4 * AS + col];
        Tq[pl - 1] = s[5 * AS + col];
        Tl[pl - 1] = s[6 * AS + col];
      }
      if (pl == 3) { T2next = s[5 * AS + col]; T2next_lo = s[6 * AS + col]; }
      if (fix && pl >= 2) fix_plane_walls<NT, BY>(s, tid, wxl, wxh, wyl, wyh, lxh, lyh);
    }
  }
  // bottom z wall inside the queue (queue slot q holds plane k0 - 2 + q);
  // constant indices keep the queues in registers
  if (wzl && k0 == 1) {
    wall_pressure(ph[2], pq[2], ph[3], pq[3], ph[1], pq[1], ph[0], pq[0]);
    wall_temperature(Tq[1], Tl[1], T2next, T2next_lo, Tq[0], Tl[0]);
  } else if (wzl && k0 == 2) {
    float hg, lg;
    wall_pressure(ph[1], pq[1], ph[2], pq[2], ph[0], pq[0], hg, lg);
  }
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f, smax = 0.f;
  bad = __syncthreads_or(bad);
  if (!bad && tid == 0) {
    // slots of planes 0 and 1 are free again
    for (; issued < min(R + 2, nplanes); ++issued) issue(issued);
  }

  for (int k = k0; k <= k1 && !bad; ++k) {
    const int pk = k - k0 + 2;  // plane index of k
    if (!wait_plane(pk + 2)) bad = true;
    if (!bad) {
      float *sk2 = slot(pk + 2);
      const float *sk = slot(pk), *sk1 = slot(pk + 1);
      ph[4] = sk2[col];
      pq[4] = sk2[AS + col];
      uq[2] = sk1[2 * AS + col];
      vq[2] = sk1[3 * AS + col];
      wq[2] = sk1[4 * AS + col];
      Tq[2] = sk1[5 * AS + col];
      Tl[2] = sk1[6 * AS + col];
      if (wzh) {
        if (k + 2 == B.nz + 1) {
          float hg, lg;
          wall_pressure(ph[3], pq[3], ph[2], pq[2], ph[4], pq[4], hg, lg);
        } else if (k + 2 == B.nz + 2) {
          extrapolate_pair(ph[3], pq[3], ph[2], pq[2], ph[4], pq[4]);  // ghost = 2 p_w - p_nz
        }
        if (k + 1 == B.nz + 1) wall_temperature(Tq[1], Tl[1], Tq[0], Tl[0], Tq[2], Tl[2]);
      }
      if (fix) fix_plane_walls<NT, BY>(sk2, tid, wxl, wxh, wyl, wyh, lxh, lyh);
      if (active) {
        const float p0h = ph[2], p0l = pq[2];
        const float *H = sk, *L = sk + AS;
        // pressure differences relative to the centre (hi/lo)
        const float axp1 = pdiff(H[col + 1], L[col + 1], p0h, p0l), axm1 = pdiff(H[col - 1], L[col - 1], p0h, p0l);
        const float axp2 = pdiff(H[col + 2], L[col + 2], p0h, p0l), axm2 = pdiff(H[col - 2], L[col - 2], p0h, p0l);
        const float ayp1 = pdiff(H[col + BX], L[col + BX], p0h, p0l), aym1 = pdiff(H[col - BX], L[col - BX], p0h, p0l);
        const float ayp2 = pdiff(H[col + 2 * BX], L[col + 2 * BX], p0h, p0l);
        const float aym2 = pdiff(H[col - 2 * BX], L[col - 2 * BX], p0h, p0l);
        const float azp1 = pdiff(ph[3], pq[3], p0h, p0l), azm1 = pdiff(ph[1], pq[1], p0h, p0l);
        const float azp2 = pdiff(ph[4], pq[4], p0h, p0l), azm2 = pdiff(ph[0], pq[0], p0h, p0l);
        const float d4x = (axp2 + axm2) - 4.f * (axp1 + axm1);
        const float d4y = (ayp2 + aym2) - 4.f * (ayp1 + aym1);
        const float d4z = (azp2 + azm2) - 4.f * (azp1 + azm1);
        const float u0 = uq[1], v0 = vq[1], w0 = wq[1], T0 = Tq[1], T0l = Tl[1];
        const float b2 = fmaxf(fmaf(u0, u0, fmaf(v0, v0, w0 * w0)), b2min);
        const float f4 = 4.f * b2;
        const float sx = fabsf(u0) + sqrt_pos(fmaf(u0, u0, f4));
        const float sy = fabsf(v0) + sqrt_pos(fmaf(v0, v0, f4));
        const float sz = fabsf(w0) + sqrt_pos(fmaf(w0, w0, f4));
        const float diss = c4h * fmaf(sx * ihx, d4x, fmaf(sy * ihy, d4y, sz * ihz * d4z));
        // transport: along each axis -V_d (q+ - q-)/(2h) + D (q+ - 2 q0 + q-)/h^2
        // = cp * (q+ - q0) + cm * (q- - q0), cp = D/h^2 - V_d/(2h), cm = D/h^2 + V_d/(2h)
        const float ax = u0 * h2x, ay = v0 * h2y, az = w0 * h2z;
        const float mpx = nhx - ax, mmx = nhx + ax, mpy = nhy - ay, mmy = nhy + ay, mpz = nhz - az, mmz = nhz + az;
        const float tpx = ahx - ax, tmx = ahx + ax, tpy = ahy - ay, tmy = ahy + ay, tpz = ahz - az, tmz = ahz + az;
        const float *Us = sk + 2 * AS, *Vs = sk + 3 * AS, *Ws = sk + 4 * AS, *Ts = sk + 5 * AS, *Tls = sk + 6 * AS;
#define BDC_F32_DIFFS(S, q0, zp, zm, dxp, dxm, dyp, dym, dzp, dzm) \
  const float dxp = S[col + 1] - q0, dxm = S[col - 1] - q0;        \
  const float dyp = S[col + BX] - q0, dym = S[col - BX] - q0;      \
  const float dzp = zp - q0, dzm = zm - q0;
        BDC_F32_DIFFS(Us, u0, uq[2], uq[0], uxp, uxm, uyp, uym, uzp, uzm)
        BDC_F32_DIFFS(Vs, v0, vq[2], vq[0], vxp, vxm, vyp, vym, vzp, vzm)
        BDC_F32_DIFFS(Ws, w0, wq[2], wq[0], wxp, wxm, wyp, wym, wzp, wzm)
#undef BDC_F32_DIFFS
        // temperature differences of the pair (hi and lo separately)
        const float txp = pdiff(Ts[col + 1], Tls[col + 1], T0, T0l), txm = pdiff(Ts[col - 1], Tls[col - 1], T0, T0l);
        const float typ = pdiff(Ts[col + BX], Tls[col + BX], T0, T0l);
        const float tym = pdiff(Ts[col - BX], Tls[col - BX], T0, T0l);
        const float tzp = pdiff(Tq[2], Tl[2], T0, T0l), tzm = pdiff(Tq[0], Tl[0], T0, T0l);
        const float tru = fmaf(mpx, uxp, fmaf(mmx, uxm, fmaf(mpy, uyp, fmaf(mmy, uym, fmaf(mpz, uzp, mmz * uzm)))));
        const float trv = fmaf(mpx, vxp, fmaf(mmx, vxm, fmaf(mpy, vyp, fmaf(mmy, vym, fmaf(mpz, vzp, mmz * vzm)))));
        const float trw = fmaf(mpx, wxp, fmaf(mmx, wxm, fmaf(mpy, wyp, fmaf(mmy, wym, fmaf(mpz, wzp, mmz * wzm)))));
        const float rT = fmaf(tpx, txp, fmaf(tmx, txm, fmaf(tpy, typ, fmaf(tmy, tym, fmaf(tpz, tzp, tmz * tzm)))));
        const float divV = fmaf(uxp - uxm, h2x, fmaf(vyp - vym, h2y, (wzp - wzm) * h2z));
        const float rp = fmaf(-b2, divV, -diss);
        const float buoy = gs * ((T0 - tinf) + T0l);
        const float ru = fmaf(-(axp1 - axm1), h2x, tru);
        const float rv = fmaf(-(ayp1 - aym1), h2y, fmaf(gy_on, buoy, trv));
        const float rw = fmaf(-(azp1 - azm1), h2z, fmaf(gz_on, buoy, trw));
        // explicit update; p and T through an error-free two-sum on their pairs
        const float un = fmaf(dt, ru, u0), vn = fmaf(dt, rv, v0), wn = fmaf(dt, rw, w0);
        float hin, lon, Tnh, Tnl;
        pair_add(p0h, p0l, fmaf(dt, rp, -cshift), hin, lon);
        pair_add(T0, T0l, dt * rT, Tnh, Tnl);
        out[0] = hin;
        out[fs] = lon;
        out[2 * fs] = un;
        out[3 * fs] = vn;
        out[4 * fs] = wn;
        out[5 * fs] = Tnh;
        out[6 * fs] = Tnl;
        s0 = fmaf(rp, rp, s0); s1 = fmaf(ru, ru, s1); s2 = fmaf(rv, rv, s2); s3 = fmaf(rw, rw, s3);
        s4 = fmaf(rT, rT, s4);
        // spectral radius of the new state: lambda_d <= |V_d| + beta gives a
        // cheap bound; the exact value is needed only where the bound could
        // raise this thread's running maximum, so the maximum is unchanged
        const float b2n = fmaxf(fmaf(un, un, fmaf(vn, vn, wn * wn)), b2min);
        const float bn = sqrt_pos(b2n);
        const float bound = fmaf(fabsf(un) + bn, ihx, fmaf(fabsf(vn) + bn, ihy, fmaf(fabsf(wn) + bn, ihz, diffsr)));
        if (bound * 1.00001f > smax) {
          const float f4n = 4.f * b2n;
          const float srn = fmaf(0.5f, fmaf(fabsf(un) + sqrt_pos(fmaf(un, un, f4n)), ihx,
                                            fmaf(fabsf(vn) + sqrt_pos(fmaf(vn, vn, f4n)), ihy,
                                                 (fabsf(wn) + sqrt_pos(fmaf(wn, wn, f4n))) * ihz)),
                                 diffsr);
          smax = fmaxf(smax, srn);
        }
      }
      out += B.plane;
      ph[0] = ph[1]; ph[1] = ph[2]; ph[2] = ph[3]; ph[3] = ph[4];
      pq[0] = pq[1]; pq[1] = pq[2]; pq[2] = pq[3]; pq[3] = pq[4];
      uq[0] = uq[1]; uq[1] = uq[2]; vq[0] = vq[1]; vq[1] = vq[2];
      wq[0] = wq[1]; wq[1] = wq[2]; Tq[0] = Tq[1]; Tq[1] = Tq[2]; Tl[0] = Tl[1]; Tl[1] = Tl[2];
    }
    bad = __syncthreads_or(bad);
    if (!bad && tid == 0 && issued < nplanes) {
      // the slot of plane pk is free: refill it with the next plane
      issue(issued);
      ++issued;
    }
  }
  if (bad) {
    // a wait gave up: record it, let this CTA's copies in flight land
    // (again bounded) before the shared memory is released
    if (tid == 0) {
      atomicOr(&a.cs[B.cav].flags, 2);
      for (int pl = max(0, issued - R); pl < issued; ++pl) (void)wait_plane(pl);
    }
    __syncthreads();
  }
  // CTA partials: FP32 per thread and per warp tree, FP64 across warps (fixed order)
  __shared__ double red[NT / 32][6];
  const int lane = tid & 31, wid = tid >> 5;
  const float w0s = warp_sum_f(s0), w1s = warp_sum_f(s1), w2s = warp_sum_f(s2), w3s = warp_sum_f(s3);
  const float w4s = warp_sum_f(s4), wms = warp_max_f(smax);
  if (lane == 0) {
    red[wid][0] = w0s; red[wid][1] = w1s; red[wid][2] = w2s; red[wid][3] = w3s; red[wid][4] = w4s;
    red[wid][5] = wms;
  }
  __syncthreads();
  if (tid < 6) {
    double acc = red[0][tid];
    for (int q = 1; q < NT / 32; ++q) acc = (tid == 5) ? fmax(acc, red[q][tid]) : acc + red[q][tid];
    a.partials[(long long)cta * kPartStride + tid] = acc;
  }
}

// Spectral-radius partials of the current state (no update), with the step
// kernel's tiling so that the finalise reduction reads the same layout.
template <class S, int TX, int TY, int KC>
__global__ void __launch_bounds__(TX *TY) k_spectral(StepArgs a) {
  constexpr int NT = TX * TY;
  const int cta = blockIdx.x;
  const int b = find_block(a.blocks, a.nblocks, cta);
  const BlockDev &B = a.blocks[b];
  const CavConst &C = a.cc[B.cav];
  const int t = cta - B.tile_begin;
  const int tx = t % B.tiles_x, ty = (t / B.tiles_x) % B.tiles_y, tz = t / (B.tiles_x * B.tiles_y);
  const int i = tx * TX + threadIdx.x + 1, j = ty * TY + threadIdx.y + 1;
  const int k0 = tz * KC + 1, k1 = min(k0 + KC - 1, B.nz);
  double smax = 0.0;
  if (i <= B.nx && j <= B.ny) {
    const S *q = (const S *)B.base[a.parity];
    const long long fs = B.fstride;
    constexpr int NP = Store<S>::NP;
    for (int k = k0; k <= k1; ++k) {
      const long long o = node_index<S>(B, i, j, k);
      smax = fmax(smax, spectral_f64(C, (double)q[NP * fs + o], (double)q[(NP + 1) * fs + o],
                                     (double)q[(NP + 2) * fs + o]));
    }
  }
  __shared__ double red[NT / 32];
  const int tid = threadIdx.y * TX + threadIdx.x;
  smax = warp_max(smax);
  if ((tid & 31) == 0) red[tid >> 5] = smax;
  __syncthreads();
  if (tid < 6) {
    double acc = 0.0;
    if (tid == 5)
      for (int q = 0; q < NT / 32; ++q) acc = fmax(acc, red[q]);
    a.partials[(long long)cta * kPartStride + tid] = acc;
  }
}

}  // namespace bdc
