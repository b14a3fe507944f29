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
// Data movement (GB300): per CTA a 32 x TY tile in (x, y) sweeps one chunk of
// its column in z, 16 x TY threads with two x-neighbouring nodes each.  One
// elected thread streams every plane of the tile with two TMA copies
// (cp.async.bulk.tensor.4d over x, y, z and the array index): the pressure
// pair with the 13-point star's halo (2 nodes in y) and u, v, w and the T
// pair with the 7-point star's (1 node in y), both 40 nodes wide (4 to the
// left of the tile: node 1 sits on a 32-byte sector boundary, so each tile's
// stores cover whole sectors, and the box starts 16-byte aligned; 4 to the
// right), into a ring of R shared-memory slots, each guarded by an mbarrier
// with a bounded wait.  A thread keeps its pair's values below the plane (z-1
// of all seven arrays, z-2 of p) in registers, so only planes k .. k+2 stay
// resident: a ring of 4 slots (47 KB) keeps one plane in flight at four CTAs
// per SM, a ring of 5 two planes at three.  HBM sees each of the seven arrays
// read once and written once per step: 56 bytes per interior point.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "bdc_device.cuh"

namespace bdc {

constexpr int kF32TX = 32;                       // tile width: 16 threads x 2 nodes
constexpr int kF32TY = 8, kF32KC = 32, kF32R = 4;  // default shape: tile height, z chunk, ring depth
constexpr int kF32HX = 4;                        // x halo of both boxes left of the tile (2 needed)
constexpr int kF32BX = kF32TX + 8;               // box width: 40 floats, 160 bytes
constexpr int kF32NA = 7;                        // p_hi, p_lo, u, v, w, T_hi, T_lo
constexpr int kF32NP = 2, kF32NO = 5;            // arrays of the pressure box and of the other box
__host__ __device__ constexpr int f32_box_yp(int TY) { return TY + 4; }  // pressure box rows: y halo 2
__host__ __device__ constexpr int f32_box_yo(int TY) { return TY + 2; }  // u, v, w, T box rows: y halo 1
__host__ __device__ constexpr int f32_p_bytes(int TY) { return kF32NP * f32_box_yp(TY) * kF32BX * 4; }
__host__ __device__ constexpr int f32_o_bytes(int TY) { return kF32NO * f32_box_yo(TY) * kF32BX * 4; }
__host__ __device__ constexpr int f32_tx_bytes(int TY) { return f32_p_bytes(TY) + f32_o_bytes(TY); }
__host__ __device__ constexpr int f32_slot_bytes(int TY) { return (f32_tx_bytes(TY) + 127) / 128 * 128; }
__host__ __device__ constexpr int f32_smem_bytes(int TY, int R) { return R * f32_slot_bytes(TY) + R * 8; }
// a box starts at node i0 - 4 (array index XO - 5 + i0, i0 = 32 t + 1): a multiple of four floats
static_assert((XO<float>::v - kF32HX) % 4 == 0, "the TMA box must start on a 16-byte boundary");
static_assert(XO<float>::v % 8 == 0, "node 1 on a 32-byte sector boundary: a tile's stores fill whole sectors");
static_assert(XO<float>::v % 2 == 0, "node pairs (odd i, i + 1) must be 8-byte aligned");
constexpr long long kWaitCycles = 4000000000LL;  // bounded mbarrier wait, about 2 s

struct StepF32Args {
  const BlockDev *blocks;
  int nblocks;
  const CavConst *cc;
  CavState *cs;               // dt and c read; flags bit 1 set on a timed-out wait
  const CUtensorMap *maps;    // [block][parity][pressure box, other box], in global memory
  double *partials;           // [slot][kPartStride]: 5 rate sums, spectral max, 2 Nusselt sums
  int parity;
  int local_dt;               // 1: each node at dt_n = cfl / S_n of its state (pseudo time)
  int ncoarse;                // coarse tiles of all blocks (scheduling indices below it)
  long long wait_cycles;      // limit of each bounded mbarrier wait (kWaitCycles)
  int withhold_plane;         // -1; a test of the timeout path sets a plane index whose load is never issued
  int ghosts_late;            // cut faces: the previous step's finalise launch writes the ghost layers
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

// wait for the phase with the given parity, giving up after `limit` cycles
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
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

// FP32 arithmetic with the rounding of every operation fixed (no contraction
// left to the compiler), on one node (float) or on two nodes packed in one
// register pair (float2: one f32x2 instruction per operation).  Both forms of
// the step kernel evaluate the same expression trees, so they give identical
// fields.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }

// f32x2 operations as PTX with an explicit rounding modifier.  The code
// generator still fuses a packed product into a packed sum that consumes
// it, so the expression trees below never add to a packed product: they use
// explicit FMAs instead, and rmul (a rounded product, per component) where
// the rounded value itself is needed (the increment of a two-sum).
#define BDC_F32X2_BINOP(NAME, OP)                                                                  \
  __device__ __forceinline__ float2 NAME(float2 a, float2 b) {                                     \
    float2 r;                                                                                      \
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t" OP \
        " rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"                                              \
        : "=f"(r.x), "=f"(r.y)                                                                     \
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                                 \
    return r;                                                                                      \
  }
BDC_F32X2_BINOP(vadd, "add.rn.f32x2")
BDC_F32X2_BINOP(vsub, "sub.rn.f32x2")
BDC_F32X2_BINOP(vmul, "mul.rn.f32x2")
#undef BDC_F32X2_BINOP
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
__device__ __forceinline__ float2 vabs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 vmax(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }

__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 rmul(float2 a, float2 b) {
  return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
}
// reciprocal square root as the one hardware approximation (relative error
// about 2^-22); its arguments here are >= kappa u_ref^2 > 0, never subnormal
__device__ __forceinline__ float vrsqrt(float a) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ float2 vrsqrt(float2 a) { return make_float2(vrsqrt(a.x), vrsqrt(a.y)); }

template <class V> __device__ __forceinline__ V splat(float s);
template <> __device__ __forceinline__ float splat<float>(float s) { return s; }
template <> __device__ __forceinline__ float2 splat<float2>(float s) { return make_float2(s, s); }

// hi/lo difference (a - c) of two FP32 pairs
template <class V>
__device__ __forceinline__ V pdiff(V ah, V al, V ch, V cl) { return vadd(vsub(ah, ch), vsub(al, cl)); }

// (h, l) + d for an FP32 pair: two-sum of the hi part, error carried into lo
template <class V>
__device__ __forceinline__ void pair_add(V h, V l, V d, V &rh, V &rl) {
  const V s = vadd(h, d);
  const V bp = vsub(s, h);
  const V e = vadd(vsub(h, vsub(s, bp)), vsub(d, bp));
  const V lo = vadd(l, e);
  rh = vadd(s, lo);
  rl = vsub(lo, vsub(rh, s));
}

__device__ __forceinline__ void split2(double v, float &hi, float &lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// a + (a - b) for FP32 pairs: the linear extrapolation 2a - b with the hi
// parts' rounding error carried into lo (two-sum), so about 48 bits survive
__device__ __forceinline__ void extrapolate_pair(float ah, float al, float bh, float bl, float &rh, float &rl) {
  const float d = vsub(ah, bh);  // exact for neighbouring values
  const float s = vadd(ah, d);
  const float bp = vsub(s, ah);
  const float e = vadd(vsub(ah, vsub(s, bp)), vsub(d, bp));
  rh = s;
  rl = vadd(e, vadd(al, vsub(al, bl)));
}

// wall and ghost pressure from the two layers next to a wall (p1 nearest):
// p_w = 2 p1 - p2, p_g = 2 p_w - p1 (one-sided second-order extrapolation)
__device__ __forceinline__ void wall_pressure(float h1, float l1, float h2, float l2, float &hw, float &lw,
                                              float &hg, float &lg) {
  extrapolate_pair(h1, l1, h2, l2, hw, lw);
  extrapolate_pair(hw, lw, h1, l1, hg, lg);
}

// adiabatic wall temperature (4 T1 - T2) / 3 = T1 + (T1 - T2) / 3 of FP32 pairs
__device__ __forceinline__ void wall_temperature(float h1, float l1, float h2, float l2, float &hw, float &lw) {
  const float d = vadd(vsub(h1, h2), vsub(l1, l2));
  pair_add(h1, l1, vmul(d, 1.f / 3.f), hw, lw);
}

// Tile of FP32 scheduling index c: coarse chunks of every block first, then
// the fine 8-plane chunks of each block's last planes (they shorten the
// grid's last wave), x tiles fastest, then y, then z.  The coarse chunk depth
// is zsplit / tiles_zc (a run-time parameter of the tiling).  The partial slot
// stays block-major (tile_begin + tx + tiles_x (ty + tiles_y tz)).
__device__ __forceinline__ TileRef f32_tile_ref(const BlockDev *blocks, int nblocks, int ncoarse, int c) {
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
  const int kc = B.zsplit / B.tiles_zc;
  TileRef T;
  T.b = lo;
  T.tx = l % B.tiles_x;
  T.ty = (l / B.tiles_x) % B.tiles_y;
  const int zl = l / (B.tiles_x * B.tiles_y);
  T.k0 = coarse ? zl * kc + 1 : B.zsplit + zl * kFineKC32 + 1;
  T.k1 = coarse ? min(T.k0 + kc - 1, B.zsplit) : min(T.k0 + kFineKC32 - 1, B.nz);
  const int tz = coarse ? zl : B.tiles_zc + zl;
  T.slot = B.tile_begin + T.tx + B.tiles_x * (T.ty + B.tiles_y * tz);
  return T;
}

// Tile of one CTA, its partial slot and the walls that fall inside its
// boxes.  Pressure box: nodes i0-4 .. i0+35, j0-2 .. j0+TY+1; other box:
// nodes i0-4 .. i0+35, j0-1 .. j0+TY; both over planes k0-2 .. k1+2 (plane
// 0 = k0-2).
struct F32Tile {
  int b, slot, i0, j0, k0, k1, tx, ty, nplanes, x0, y0, zbase, lxh, lyh;
  bool wxl, wxh, wyl, wyh, wzl, wzh, fix;
};

template <int TY>
__device__ __forceinline__ F32Tile f32_tile(const StepF32Args &a, int cta) {
  F32Tile T;
  const TileRef R = f32_tile_ref(a.blocks, a.nblocks, a.ncoarse, cta);
  T.b = R.b;
  T.slot = R.slot;
  const BlockDev &B = a.blocks[T.b];
  T.tx = R.tx;
  T.ty = R.ty;
  T.i0 = T.tx * kF32TX + 1;
  T.j0 = T.ty * TY + 1;
  T.k0 = R.k0;
  T.k1 = R.k1;
  T.nplanes = (T.k1 - T.k0 + 1) + 4;       // z = k0-2 .. k1+2
  T.x0 = XO<float>::v - 1 + T.i0 - kF32HX;  // array index of node i0 - 4
  T.y0 = (T.j0 - 2) + 1;                    // array row of node j0 - 2 (the pressure box)
  T.zbase = (T.k0 - 2) + 1;                 // array plane of the tile's plane 0
  T.wxl = B.wall[0] && T.tx == 0;
  T.wxh = B.wall[1] && B.nx + 1 <= T.i0 + kF32TX + 3;  // the wall node nx + 1 inside the boxes
  T.wyl = B.wall[2] && T.ty == 0;
  T.wyh = B.wall[3] && B.ny + 1 <= T.j0 + TY + 1;      // the wall node ny + 1 inside the pressure box
  T.wzl = B.wall[4];
  T.wzh = B.wall[5];
  T.fix = T.wxl || T.wxh || T.wyl || T.wyh;
  T.lxh = B.nx - T.i0 + kF32HX;  // box column of node nx
  T.lyh = B.ny - T.j0 + 2;       // pressure-box row of node ny (other box: one row less)
  return T;
}

// Whether the tile's boxes (x nodes i0-4 .. i0+35, y rows j0-2 .. j0+TY+1,
// planes k0-2 .. k1+2) reach a ghost layer of a cut face.
template <int TY>
__device__ __forceinline__ bool f32_reads_ghosts(const BlockDev &B, const F32Tile &T) {
  return (!B.wall[0] && T.i0 - kF32HX <= 0) || (!B.wall[1] && T.i0 + kF32BX - kF32HX - 1 >= B.nx + 1) ||
         (!B.wall[2] && T.j0 - 2 <= 0) || (!B.wall[3] && T.j0 + TY + 1 >= B.ny + 1) ||
         (!B.wall[4] && T.k0 - 2 <= 0) || (!B.wall[5] && T.k1 + 2 >= B.nz + 1);
}

// Apply the x and y wall conditions to one freshly loaded plane slot.
// Pressure-box coordinates: column i - i0 + 4, row j - j0 + 2; other box:
// the same columns, row j - j0 + 1.  Threads [0, BX) take the low y wall,
// [BX, 2BX) the high y wall, the next BYP the low x wall and the next BYP the
// high x wall (x walls: pressure only; their temperature is prescribed and
// stored).  Groups that read a corner another group writes only produce
// corner values, which no star stencil reads.
template <int NT, int TY>
__device__ __forceinline__ void fix_plane_walls(float *s, int tid, const F32Tile &T) {
  constexpr int BX = kF32BX, BYP = f32_box_yp(TY), BYO = f32_box_yo(TY);
  constexpr int APS = BX * BYP, AOS = BX * BYO;
  float *H = s, *L = s + APS;                    // p pair
  float *TH = s + 2 * APS + 3 * AOS, *TL = TH + AOS;  // T pair
  static_assert(NT >= 2 * (BX + BYP), "thread groups");
  float hw, lw, hg, lg;
  if (T.wyl && tid < BX) {
    const int x = tid;
    // nodes 1, 2 at pressure rows 2, 3: wall (row 1) and ghost (row 0)
    wall_pressure(H[2 * BX + x], L[2 * BX + x], H[3 * BX + x], L[3 * BX + x], hw, lw, hg, lg);
    H[BX + x] = hw; L[BX + x] = lw; H[x] = hg; L[x] = lg;
    // nodes 1, 2 at rows 1, 2 of the other box: wall at row 0
    wall_temperature(TH[BX + x], TL[BX + x], TH[2 * BX + x], TL[2 * BX + x], TH[x], TL[x]);
  } else if (T.wyh && tid >= BX && tid < 2 * BX) {
    const int x = tid - BX;
    const int r1 = T.lyh, r2 = r1 - 1;  // pressure rows of nodes ny and ny - 1
    wall_pressure(H[r1 * BX + x], L[r1 * BX + x], H[r2 * BX + x], L[r2 * BX + x], hw, lw, hg, lg);
    H[(r1 + 1) * BX + x] = hw; L[(r1 + 1) * BX + x] = lw;
    if (r1 + 2 < BYP) { H[(r1 + 2) * BX + x] = hg; L[(r1 + 2) * BX + x] = lg; }
    const int o1 = r1 - 1;  // other-box row of node ny
    if (o1 + 1 < BYO)
      wall_temperature(TH[o1 * BX + x], TL[o1 * BX + x], TH[(o1 - 1) * BX + x], TL[(o1 - 1) * BX + x],
                       TH[(o1 + 1) * BX + x], TL[(o1 + 1) * BX + x]);
  } else if (T.wxl && tid >= 2 * BX && tid < 2 * BX + BYP) {
    const int y = tid - 2 * BX;
    // nodes 1, 2 at columns 4, 5: wall (column 3) and ghost (column 2)
    constexpr int c1 = kF32HX;
    wall_pressure(H[y * BX + c1], L[y * BX + c1], H[y * BX + c1 + 1], L[y * BX + c1 + 1], hw, lw, hg, lg);
    H[y * BX + c1 - 1] = hw; L[y * BX + c1 - 1] = lw; H[y * BX + c1 - 2] = hg; L[y * BX + c1 - 2] = lg;
  } else if (T.wxh && tid >= 2 * BX + BYP && tid < 2 * (BX + BYP)) {
    const int y = tid - 2 * BX - BYP;
    const int c1 = T.lxh, c2 = c1 - 1;  // columns of nodes nx and nx - 1
    wall_pressure(H[y * BX + c1], L[y * BX + c1], H[y * BX + c2], L[y * BX + c2], hw, lw, hg, lg);
    H[y * BX + c1 + 1] = hw; L[y * BX + c1 + 1] = lw;
    if (c1 + 2 < BX) { H[y * BX + c1 + 2] = hg; L[y * BX + c1 + 2] = lg; }
  }
  // the slot is refilled by TMA later: order these generic-proxy writes
  // before the async proxy's
  if (tid < 2 * (BX + BYP)) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

// Constants of the FP32 update, broadcast to the value type.
template <class V>
struct F32K {
  V ihx, ihy, ihz, h2x, h2y, h2z, mh2x, mh2y, mh2z, nhx, nhy, nhz, ahx, ahy, ahz, c4h, gs, tinf, b2min, dt, mdt, mcs, gy,
      gz, diffsr, cfl;
};

template <class V>
__device__ __forceinline__ F32K<V> f32_consts(const CavConst &C, const CavState &S) {
  F32K<V> K;
  // the static constants come rounded to FP32 from the host; only dt and the
  // centre shift are converted here
  K.ihx = splat<V>(C.fih[0]); K.ihy = splat<V>(C.fih[1]); K.ihz = splat<V>(C.fih[2]);
  K.h2x = splat<V>(C.fh2[0]); K.h2y = splat<V>(C.fh2[1]); K.h2z = splat<V>(C.fh2[2]);
  K.mh2x = splat<V>(-C.fh2[0]); K.mh2y = splat<V>(-C.fh2[1]); K.mh2z = splat<V>(-C.fh2[2]);
  K.nhx = splat<V>(C.fnh[0]); K.nhy = splat<V>(C.fnh[1]); K.nhz = splat<V>(C.fnh[2]);
  K.ahx = splat<V>(C.fah[0]); K.ahy = splat<V>(C.fah[1]); K.ahz = splat<V>(C.fah[2]);
  K.c4h = splat<V>(C.fc4h); K.gs = splat<V>(C.fgs); K.tinf = splat<V>(C.ftinf);
  K.b2min = splat<V>(C.fb2min);
  const float dt = (float)S.dt;
  K.dt = splat<V>(dt); K.mdt = splat<V>(-dt); K.mcs = splat<V>(-(float)S.c);
  K.gy = splat<V>(C.gaxis == 1 ? 1.f : 0.f); K.gz = splat<V>(C.gaxis == 2 ? 1.f : 0.f);
  K.diffsr = splat<V>(C.fdiffsr);
  K.cfl = splat<V>(C.fcfl);
  return K;
}

// The stencil of one node (or two): centre values and neighbour-minus-centre
// differences (hi/lo pair differences for p and T).
template <class V>
struct F32Nb {
  V ph, pl;                                                                  // centre p pair
  V pxp1, pxm1, pxp2, pxm2, pyp1, pym1, pyp2, pym2, pzp1, pzm1, pzp2, pzm2;  // p differences
  V u, v, w, th, tl;                                                         // centre u, v, w, T pair
  V uxp, uxm, uyp, uym, uzp, uzm, vxp, vxm, vyp, vym, vzp, vzm, wxp, wxm, wyp, wym, wzp, wzm;
  V txp, txm, typ, tym, tzp, tzm;
};

template <class V>
struct F32Out {
  V ph, pl, u, v, w, th, tl;  // new state
  V rp, ru, rv, rw, rt;       // rates (rp with the sign flipped; only its square is summed)
};

// Rates of Eqs. 1-3 at the node(s) and the explicit update with step dt
// (mdt = -dt); p and T through an error-free two-sum on their pairs.
template <class V>
__device__ __forceinline__ void f32_update(const F32K<V> &K, const F32Nb<V> &n, V dt, V mdt, F32Out<V> &o) {
  const V m4 = splat<V>(-4.f), four = splat<V>(4.f);
  const V d4x = vfma(m4, vadd(n.pxp1, n.pxm1), vadd(n.pxp2, n.pxm2));
  const V d4y = vfma(m4, vadd(n.pyp1, n.pym1), vadd(n.pyp2, n.pym2));
  const V d4z = vfma(m4, vadd(n.pzp1, n.pzm1), vadd(n.pzp2, n.pzm2));
  const V b2 = vmax(vfma(n.u, n.u, vfma(n.v, n.v, vmul(n.w, n.w))), K.b2min);
  const V f4 = vmul(four, b2);
  // 2 lambda_d = |V_d| + sqrt(V_d^2 + 4 beta^2), the root as x * rsqrt(x) fused
  const V qx = vfma(n.u, n.u, f4), qy = vfma(n.v, n.v, f4), qz = vfma(n.w, n.w, f4);
  const V sx = vfma(qx, vrsqrt(qx), vabs(n.u));
  const V sy = vfma(qy, vrsqrt(qy), vabs(n.v));
  const V sz = vfma(qz, vrsqrt(qz), vabs(n.w));
  const V diss = vmul(K.c4h, vfma(vmul(sx, K.ihx), d4x, vfma(vmul(sy, K.ihy), d4y, vmul(vmul(sz, K.ihz), d4z))));
  // transport: along each axis -V_d (q+ - q-)/(2h) + D (q+ - 2 q0 + q-)/h^2
  // = cp * (q+ - q0) + cm * (q- - q0), cp = D/h^2 - V_d/(2h), cm = D/h^2 + V_d/(2h)
  const V mpx = vfma(n.u, K.mh2x, K.nhx), mmx = vfma(n.u, K.h2x, K.nhx);
  const V mpy = vfma(n.v, K.mh2y, K.nhy), mmy = vfma(n.v, K.h2y, K.nhy);
  const V mpz = vfma(n.w, K.mh2z, K.nhz), mmz = vfma(n.w, K.h2z, K.nhz);
  const V tpx = vfma(n.u, K.mh2x, K.ahx), tmx = vfma(n.u, K.h2x, K.ahx);
  const V tpy = vfma(n.v, K.mh2y, K.ahy), tmy = vfma(n.v, K.h2y, K.ahy);
  const V tpz = vfma(n.w, K.mh2z, K.ahz), tmz = vfma(n.w, K.h2z, K.ahz);
  const V tru = vfma(mpx, n.uxp, vfma(mmx, n.uxm, vfma(mpy, n.uyp, vfma(mmy, n.uym, vfma(mpz, n.uzp, vmul(mmz, n.uzm))))));
  const V trv = vfma(mpx, n.vxp, vfma(mmx, n.vxm, vfma(mpy, n.vyp, vfma(mmy, n.vym, vfma(mpz, n.vzp, vmul(mmz, n.vzm))))));
  const V trw = vfma(mpx, n.wxp, vfma(mmx, n.wxm, vfma(mpy, n.wyp, vfma(mmy, n.wym, vfma(mpz, n.wzp, vmul(mmz, n.wzm))))));
  o.rt = vfma(tpx, n.txp, vfma(tmx, n.txm, vfma(tpy, n.typ, vfma(tmy, n.tym, vfma(tpz, n.tzp, vmul(tmz, n.tzm))))));
  const V divV = vfma(vsub(n.uxp, n.uxm), K.h2x, vfma(vsub(n.vyp, n.vym), K.h2y, vmul(vsub(n.wzp, n.wzm), K.h2z)));
  o.rp = vfma(b2, divV, diss);  // = -dp/dt
  const V buoy = vmul(K.gs, vadd(vsub(n.th, K.tinf), n.tl));
  o.ru = vfma(vsub(n.pxm1, n.pxp1), K.h2x, tru);
  o.rv = vfma(vsub(n.pym1, n.pyp1), K.h2y, vfma(K.gy, buoy, trv));
  o.rw = vfma(vsub(n.pzm1, n.pzp1), K.h2z, vfma(K.gz, buoy, trw));
  o.u = vfma(dt, o.ru, n.u);
  o.v = vfma(dt, o.rv, n.v);
  o.w = vfma(dt, o.rw, n.w);
  pair_add(n.ph, n.pl, vfma(mdt, o.rp, K.mcs), o.ph, o.pl);  // p - dt (-dp/dt) - pending centre shift
  pair_add(n.th, n.tl, rmul(dt, o.rt), o.th, o.tl);
}

// Spectral radius of the new state: lambda_d <= |V_d| + beta gives a cheap
// bound; the exact value is needed only where the bound could raise the
// thread's running maximum, so the maximum is unchanged.
template <class V>
__device__ __forceinline__ V f32_spectral_bound(const F32K<V> &K, V un, V vn, V wn) {
  const V b2n = vmax(vfma(un, un, vfma(vn, vn, vmul(wn, wn))), K.b2min);
  const V rb = vrsqrt(b2n);  // beta = b2n * rsqrt(b2n), fused into each |V_d| + beta
  return vfma(vfma(b2n, rb, vabs(un)), K.ihx, vfma(vfma(b2n, rb, vabs(vn)), K.ihy, vfma(vfma(b2n, rb, vabs(wn)), K.ihz, K.diffsr)));
}

__device__ __forceinline__ float f32_spectral_exact(const F32K<float> &K, float un, float vn, float wn) {
  const float b2n = vmax(vfma(un, un, vfma(vn, vn, vmul(wn, wn))), K.b2min);
  const float f4n = vmul(4.f, b2n);
  const float qx = vfma(un, un, f4n), qy = vfma(vn, vn, f4n), qz = vfma(wn, wn, f4n);
  const float sx = vfma(qx, vrsqrt(qx), vabs(un));
  const float sy = vfma(qy, vrsqrt(qy), vabs(vn));
  const float sz = vfma(qz, vrsqrt(qz), vabs(wn));
  return vfma(0.5f, vfma(sx, K.ihx, vfma(sy, K.ihy, vmul(sz, K.ihz))), K.diffsr);
}

// the constants f32_spectral_exact reads (beta_min^2, 1/h, the diffusive term)
__device__ __forceinline__ F32K<float> f32_spectral_consts(const CavConst &C) {
  F32K<float> K{};
  K.b2min = C.fb2min;
  K.ihx = C.fih[0];
  K.ihy = C.fih[1];
  K.ihz = C.fih[2];
  K.diffsr = C.fdiffsr;
  return K;
}

__device__ __forceinline__ void f32_spectral_max(const F32K<float> &K, float bound, float un, float vn, float wn,
                                                 float &smax) {
  if (vmul(bound, 1.00001f) > smax) smax = fmaxf(smax, f32_spectral_exact(K, un, vn, wn));
}

// CTA partials: rate sums FP32 per thread and per warp tree, FP64 across
// warps (fixed order); Nusselt sums FP64 from the column sums on.  Slots:
// 5 rate sums, spectral max, hot and cold sums of 3 T_w - 4 T_1 + T_2; the
// per-cavity reduction (k_finalize) reads them in a fixed order.
// `xwall`: the tile touches an isothermal x wall (uniform over the CTA); only
// then can a thread hold Nusselt sums, and the FP64 warp sums run.
template <int NT>
__device__ __forceinline__ void f32_partials(double *partials, int cta, int tid, float s0, float s1, float s2,
                                             float s3, float s4, float smax, double nuh, double nuc, bool xwall) {
  __shared__ double red[NT / 32][8];
  const int lane = tid & 31, wid = tid >> 5;
  const float w0s = warp_sum_f(s0), w1s = warp_sum_f(s1), w2s = warp_sum_f(s2), w3s = warp_sum_f(s3);
  const float w4s = warp_sum_f(s4), wms = warp_max_f(smax);
  const double wnh = xwall ? warp_sum(nuh) : 0.0, wnc = xwall ? warp_sum(nuc) : 0.0;
  if (lane == 0) {
    red[wid][0] = w0s; red[wid][1] = w1s; red[wid][2] = w2s; red[wid][3] = w3s; red[wid][4] = w4s;
    red[wid][5] = wms; red[wid][6] = wnh; red[wid][7] = wnc;
  }
  __syncthreads();
  if (tid < 8) {
    double acc = red[0][tid];
    for (int q = 1; q < NT / 32; ++q) acc = (tid == 5) ? fmax(acc, red[q][tid]) : acc + red[q][tid];
    partials[(long long)cta * kPartStride + tid] = acc;
  }
}

__device__ __forceinline__ double pair_value(float h, float l) { return (double)h + (double)l; }

// (sh, sl) += (h, l): compensated FP32 sum (two-sum of the hi parts).  The
// Nusselt sums use it for the columns next to an isothermal x wall: the sum
// over a column's chunk of the new T (and of the stored wall T beside it)
// keeps about 48 bits, and 3 T_w - 4 T_1 + T_2 is formed from those sums in
// FP64 after the sweep, so no FP64 work runs per node.
template <class V>
__device__ __forceinline__ void acc_pair(V &sh, V &sl, V h, V l) {
  const V s = vadd(sh, h);
  const V bp = vsub(s, sh);
  const V e = vadd(vsub(sh, vsub(s, bp)), vsub(h, bp));
  sl = vadd(sl, vadd(e, l));
  sh = s;
}

__device__ __forceinline__ float2 ld2(const float *s, int idx) { return *reinterpret_cast<const float2 *>(s + idx); }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
// Per-thread state of the FP32 step kernel (two nodes per thread):
// the pair's z - 1 values of all seven arrays and p's z - 2 values, the
// running residual sums and spectral maximum, and the Nusselt column sums.
struct F32QAcc {
  float2 qm1[7], qm2h, qm2l;
  float2 s0, s1, s2, s3, s4;
  float smax;
  float2 ch, cl;
  float wsh, wsl;
  float wch, wcl;  // the cold wall's T when the pair also borders the hot wall (nx = 2)
};

// One plane of one thread's node pair: rates and update of the pair at plane
// k from the resident slots of planes k, k+1, k+2 (S0, Sp1, Sp2) and the
// register queues (planes k-1, k-2); writes the new state at `out`,
// accumulates the sums and moves the queues one plane up.  `colp` / `col`:
// the pair's first node in the pressure box / the other box of a slot;
// `wofs`: offset of the wall value read for the Nusselt sum.
template <int TY>
__device__ __forceinline__ void f32q_pair(const float *S0, const float *Sp1, const float *Sp2, const F32K<float2> &K,
                                          const F32K<float> &K1, int k, int nz, bool wzl, bool wzh, int local_dt,
                                          float *out, long long fs, int colp, int col, int wofs, bool act1,
                                          bool nus_warp, F32QAcc &acc) {
  constexpr int BX = kF32BX, APS = BX * f32_box_yp(TY), AOS = BX * f32_box_yo(TY);
  constexpr int OO = 2 * APS;            // the other box inside a slot: u, v, w, T_hi, T_lo
  constexpr int TO = OO + 3 * AOS;       // T_hi inside a slot
  float2(&qm1)[7] = acc.qm1;
  float2 &qm2h = acc.qm2h, &qm2l = acc.qm2l;
  float2 &s0 = acc.s0, &s1 = acc.s1, &s2 = acc.s2, &s3 = acc.s3, &s4 = acc.s4;
  float &smax = acc.smax;
  float2 &ch = acc.ch, &cl = acc.cl;
  float &wsh = acc.wsh, &wsl = acc.wsl;
  F32Nb<float2> n;
  // pressure: centre pair and its z neighbours (walls formed in place)
  n.ph = ld2(S0, colp);
  n.pl = ld2(S0 + APS, colp);
  float2 zm2h = qm2h, zm2l = qm2l, zm1h = qm1[0], zm1l = qm1[1];
  float2 zp1h = ld2(Sp1, colp), zp1l = ld2(Sp1 + APS, colp), zp2h = ld2(Sp2, colp), zp2l = ld2(Sp2 + APS, colp);
  float2 th = ld2(S0 + TO, col), tl = ld2(S0 + TO + AOS, col);
  float2 tzmh = qm1[5], tzml = qm1[6];
  float2 tzph = ld2(Sp1 + TO, col), tzpl = ld2(Sp1 + TO + AOS, col);
  if (wzl && k <= 2) {
    float hg, lg;
    if (k == 1) {  // z = 0 wall and z = -1 ghost from the layers z = 1, 2
      wall_pressure(n.ph.x, n.pl.x, zp1h.x, zp1l.x, zm1h.x, zm1l.x, zm2h.x, zm2l.x);
      wall_pressure(n.ph.y, n.pl.y, zp1h.y, zp1l.y, zm1h.y, zm1l.y, zm2h.y, zm2l.y);
      wall_temperature(th.x, tl.x, tzph.x, tzpl.x, tzmh.x, tzml.x);
      wall_temperature(th.y, tl.y, tzph.y, tzpl.y, tzmh.y, tzml.y);
    } else {  // k == 2: z = 0 wall from z = 1, 2
      wall_pressure(zm1h.x, zm1l.x, n.ph.x, n.pl.x, zm2h.x, zm2l.x, hg, lg);
      wall_pressure(zm1h.y, zm1l.y, n.ph.y, n.pl.y, zm2h.y, zm2l.y, hg, lg);
    }
  }
  if (wzh && k >= nz - 1) {
    float hg, lg;
    if (k == nz) {  // z = nz+1 wall and nz+2 ghost from the layers nz, nz-1
      wall_pressure(n.ph.x, n.pl.x, zm1h.x, zm1l.x, zp1h.x, zp1l.x, zp2h.x, zp2l.x);
      wall_pressure(n.ph.y, n.pl.y, zm1h.y, zm1l.y, zp1h.y, zp1l.y, zp2h.y, zp2l.y);
      wall_temperature(th.x, tl.x, tzmh.x, tzml.x, tzph.x, tzpl.x);
      wall_temperature(th.y, tl.y, tzmh.y, tzml.y, tzph.y, tzpl.y);
    } else {  // k == nz-1: z = nz+1 wall from nz, nz-1
      wall_pressure(zp1h.x, zp1l.x, n.ph.x, n.pl.x, zp2h.x, zp2l.x, hg, lg);
      wall_pressure(zp1h.y, zp1l.y, n.ph.y, n.pl.y, zp2h.y, zp2l.y, hg, lg);
    }
  }
  n.pzp1 = pdiff(zp1h, zp1l, n.ph, n.pl);
  n.pzm1 = pdiff(zm1h, zm1l, n.ph, n.pl);
  n.pzp2 = pdiff(zp2h, zp2l, n.ph, n.pl);
  n.pzm2 = pdiff(zm2h, zm2l, n.ph, n.pl);
  {
    const float *H = S0, *L = S0 + APS;
    const float2 ah = ld2(H, colp - 2), al = ld2(L, colp - 2), dh = ld2(H, colp + 2), dl = ld2(L, colp + 2);
    n.pxp1 = make_float2(pdiff(n.ph.y, n.pl.y, n.ph.x, n.pl.x), pdiff(dh.x, dl.x, n.ph.y, n.pl.y));
    n.pxm1 = make_float2(pdiff(ah.y, al.y, n.ph.x, n.pl.x), pdiff(n.ph.x, n.pl.x, n.ph.y, n.pl.y));
    n.pxp2 = pdiff(dh, dl, n.ph, n.pl);
    n.pxm2 = pdiff(ah, al, n.ph, n.pl);
    n.pyp1 = pdiff(ld2(H, colp + BX), ld2(L, colp + BX), n.ph, n.pl);
    n.pym1 = pdiff(ld2(H, colp - BX), ld2(L, colp - BX), n.ph, n.pl);
    n.pyp2 = pdiff(ld2(H, colp + 2 * BX), ld2(L, colp + 2 * BX), n.ph, n.pl);
    n.pym2 = pdiff(ld2(H, colp - 2 * BX), ld2(L, colp - 2 * BX), n.ph, n.pl);
  }
  // velocity: x differences per node, y and z packed
#define BDC_F32Q_VEL(F, c0, xp, xm, yp, ym, zp, zm)                                                  \
  {                                                                                                \
    const float *Q = S0 + OO + (F - 2) * AOS;                                                      \
    c0 = ld2(Q, col);                                                                              \
    const float qm = Q[col - 1], qp = Q[col + 2];                                                  \
    xp = make_float2(vsub(c0.y, c0.x), vsub(qp, c0.y));                                            \
    xm = make_float2(vsub(qm, c0.x), vsub(c0.x, c0.y));                                            \
    yp = vsub(ld2(Q, col + BX), c0);                                                               \
    ym = vsub(ld2(Q, col - BX), c0);                                                               \
    zp = vsub(ld2(Sp1 + OO + (F - 2) * AOS, col), c0);                                             \
    zm = vsub(qm1[F], c0);                                                                         \
  }
  BDC_F32Q_VEL(2, n.u, n.uxp, n.uxm, n.uyp, n.uym, n.uzp, n.uzm)
  BDC_F32Q_VEL(3, n.v, n.vxp, n.vxm, n.vyp, n.vym, n.vzp, n.vzm)
  BDC_F32Q_VEL(4, n.w, n.wxp, n.wxm, n.wyp, n.wym, n.wzp, n.wzm)
#undef BDC_F32Q_VEL
  // temperature pair
  n.th = th;
  n.tl = tl;
  {
    const float *TH = S0 + TO, *TL = S0 + TO + AOS;
    n.txp = make_float2(pdiff(th.y, tl.y, th.x, tl.x), pdiff(TH[col + 2], TL[col + 2], th.y, tl.y));
    n.txm = make_float2(pdiff(TH[col - 1], TL[col - 1], th.x, tl.x), pdiff(th.x, tl.x, th.y, tl.y));
    n.typ = pdiff(ld2(TH, col + BX), ld2(TL, col + BX), th, tl);
    n.tym = pdiff(ld2(TH, col - BX), ld2(TL, col - BX), th, tl);
    n.tzp = pdiff(tzph, tzpl, th, tl);
    n.tzm = pdiff(tzmh, tzml, th, tl);
  }
  F32Out<float2> o;
  float2 dtn = K.dt, mdtn = K.mdt;
  if (local_dt) {  // each node's own stable step
    dtn = make_float2(__fdiv_rn(K1.cfl, f32_spectral_exact(K1, n.u.x, n.v.x, n.w.x)),
                      __fdiv_rn(K1.cfl, f32_spectral_exact(K1, n.u.y, n.v.y, n.w.y)));
    mdtn = make_float2(-dtn.x, -dtn.y);
  }
  f32_update(K, n, dtn, mdtn, o);
  const float2 bound = f32_spectral_bound(K, o.u, o.v, o.w);
  f32_spectral_max(K1, bound.x, o.u.x, o.v.x, o.w.x, smax);
  if (act1) {
    st2(out, o.ph);
    st2(out + fs, o.pl);
    st2(out + 2 * fs, o.u);
    st2(out + 3 * fs, o.v);
    st2(out + 4 * fs, o.w);
    st2(out + 5 * fs, o.th);
    st2(out + 6 * fs, o.tl);
    f32_spectral_max(K1, bound.y, o.u.y, o.v.y, o.w.y, smax);
  } else {  // the x extent is odd: the pair's second node is a wall or beyond
    out[0] = o.ph.x;
    out[fs] = o.pl.x;
    out[2 * fs] = o.u.x;
    out[3 * fs] = o.v.x;
    out[4 * fs] = o.w.x;
    out[5 * fs] = o.th.x;
    out[6 * fs] = o.tl.x;
    o.rp.y = o.ru.y = o.rv.y = o.rw.y = o.rt.y = 0.f;
  }
  s0 = vfma(o.rp, o.rp, s0); s1 = vfma(o.ru, o.ru, s1); s2 = vfma(o.rv, o.rv, s2);
  s3 = vfma(o.rw, o.rw, s3); s4 = vfma(o.rt, o.rt, s4);
  if (nus_warp) {
    acc_pair(ch, cl, o.th, o.tl);
    acc_pair(wsh, wsl, S0[TO + col + wofs], S0[TO + AOS + col + wofs]);
    // a pair (1, 2) with nx = 2 borders both x walls: the cold wall is node 3
    if (wofs == -1) acc_pair(acc.wch, acc.wcl, S0[TO + col + 2], S0[TO + AOS + col + 2]);
  }
  // the register queues move one plane: z - 2 <- z - 1 (p), z - 1 <- this plane
  qm2h = qm1[0];
  qm2l = qm1[1];
  qm1[0] = n.ph; qm1[1] = n.pl; qm1[2] = n.u; qm1[3] = n.v; qm1[4] = n.w; qm1[5] = th; qm1[6] = tl;
}

// The node pair of one thread in a tile and its Nusselt weights (the two
// columns' weights in 3 T_w - 4 T_1 + T_2).
struct F32QCol {
  int i, j, colp, col, wofs;
  bool act0, act1, nus, nus_warp, hot_next, cold_next;
  double wh0, wh1, wc0, wc1;
};

// Called by every thread of the CTA (a warp vote).
__device__ __forceinline__ F32QCol f32q_column(const BlockDev &B, const F32Tile &T, int li, int lj) {
  F32QCol c;
  const int i = T.i0 + 2 * li, j = T.j0 + lj;
  c.i = i;
  c.j = j;
  c.act0 = (i <= B.nx) && (j <= B.ny);
  c.act1 = (i + 1 <= B.nx) && (j <= B.ny);
  const bool xw0 = B.wall[0], xw1 = B.wall[1];
  c.wh0 = (xw0 && c.act0) ? (i == 1 ? -4.0 : (i == 2 ? 1.0 : 0.0)) : 0.0;
  c.wh1 = (xw0 && c.act1) ? (i + 1 == 2 ? 1.0 : 0.0) : 0.0;
  c.wc0 = (xw1 && c.act0) ? (i == B.nx ? -4.0 : (i == B.nx - 1 ? 1.0 : 0.0)) : 0.0;
  c.wc1 = (xw1 && c.act1) ? (i + 1 == B.nx ? -4.0 : (i + 1 == B.nx - 1 ? 1.0 : 0.0)) : 0.0;
  c.nus = (xw0 && c.act0 && i <= 2) || (xw0 && c.act1 && i + 1 == 2) || (xw1 && c.act0 && i >= B.nx - 1) ||
          (xw1 && c.act1 && i + 1 >= B.nx - 1);
  // the column beside a wall: node i next to x = 0 or x = nx + 1, or node i + 1 next to x = nx + 1
  c.hot_next = xw0 && c.act0 && i == 1;
  const bool cold_next0 = xw1 && c.act0 && i == B.nx, cold_next1 = xw1 && c.act1 && i + 1 == B.nx;
  c.cold_next = cold_next0 || cold_next1;
  c.wofs = c.hot_next ? -1 : (cold_next0 ? 1 : 2);
  c.nus_warp = __any_sync(0xffffffffu, c.nus);
  // the pair's first node in the pressure box and in the other box (even: 8-byte aligned)
  c.colp = (lj + 2) * kF32BX + (2 * li + kF32HX);
  c.col = (lj + 1) * kF32BX + (2 * li + kF32HX);
  return c;
}

__device__ __forceinline__ void f32q_clear(F32QAcc &acc) {
  const float2 z = make_float2(0.f, 0.f);
  for (int q = 0; q < 7; ++q) acc.qm1[q] = z;
  acc.qm2h = acc.qm2l = z;
  acc.s0 = acc.s1 = acc.s2 = acc.s3 = acc.s4 = z;
  acc.smax = 0.f;
  acc.ch = acc.cl = z;
  acc.wsh = acc.wsl = 0.f;
  acc.wch = acc.wcl = 0.f;
}

// The tile's partials (every thread of the CTA calls it: a CTA reduction).
template <int NT>
__device__ __forceinline__ void f32q_finish(double *partials, int tile, int tid, const F32Tile &T, const F32QCol &c,
                                            const F32QAcc &acc) {
  double nuh = 0.0, nuc = 0.0;
  if (c.nus) {
    const double t0 = pair_value(acc.ch.x, acc.cl.x), t1 = c.act1 ? pair_value(acc.ch.y, acc.cl.y) : 0.0;
    const double wall_t = 3.0 * pair_value(acc.wsh, acc.wsl);
    // the cold wall's sum: the second accumulator where the pair borders both walls
    const double wall_c = c.hot_next ? 3.0 * pair_value(acc.wch, acc.wcl) : wall_t;
    nuh = c.wh0 * t0 + c.wh1 * t1 + (c.hot_next ? wall_t : 0.0);
    nuc = c.wc0 * t0 + c.wc1 * t1 + (c.cold_next ? wall_c : 0.0);
  }
  f32_partials<NT>(partials, tile, tid, vadd(acc.s0.x, acc.s0.y), vadd(acc.s1.x, acc.s1.y), vadd(acc.s2.x, acc.s2.y),
                   vadd(acc.s3.x, acc.s3.y), vadd(acc.s4.x, acc.s4.y), acc.smax, nuh, nuc, T.wxl || T.wxh);
}

// The tile's prologue reads once planes 0 .. 3 (z = k0-2 .. k0+1) are resident
// in their slots: the x and y walls of the interior planes 2 and 3 are formed
// in place, and the register queues take plane 1 (z - 1, seven arrays) and
// plane 0 (z - 2, p).
template <int NT, int TY>
__device__ __forceinline__ void f32q_prologue_plane(int pl, float *S, const F32Tile &T, const F32QCol &c, int tid,
                                                    F32QAcc &acc) {
  constexpr int APS = kF32BX * f32_box_yp(TY), AOS = kF32BX * f32_box_yo(TY);
  if (T.fix && pl >= 2) fix_plane_walls<NT, TY>(S, tid, T);
  if (c.act0 && pl == 0) {
    acc.qm2h = ld2(S, c.colp);
    acc.qm2l = ld2(S + APS, c.colp);
  }
  if (c.act0 && pl == 1) {
    acc.qm1[0] = ld2(S, c.colp);
    acc.qm1[1] = ld2(S + APS, c.colp);
    for (int q = 2; q < 7; ++q) acc.qm1[q] = ld2(S + 2 * APS + (q - 2) * AOS, c.col);
  }
}

// The fused FP32-mixed step: one CTA per tile (a 32 x TY tile of nodes, one
// z chunk of its column), 16 x TY threads with two nodes each.  Planes arrive
// in a ring of R slots: the slot of plane p is refilled with
// plane p + R once plane p is done, so with three planes resident R - 3
// planes are in flight.  R = 4 at 47 KB per CTA keeps one plane in flight
// with four CTAs (16 warps) per SM, R = 5 at 59 KB two planes with three; the
// launch bounds ask for 512 threads per SM, which the compiler meets in at
// most 128 registers.
template <int TY, int R>
__global__ void __launch_bounds__(kF32TX / 2 * TY, 512 / (kF32TX / 2 * TY)) k_step_f32q(StepF32Args a) {
  static_assert(R >= 4, "ring depth: three planes resident and at least one in flight");
  constexpr int NTX = kF32TX / 2, NT = NTX * TY;
  constexpr int SB = f32_slot_bytes(TY), SF = SB / 4, PF = f32_p_bytes(TY) / 4;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float *ring = reinterpret_cast<float *>(smem_raw);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + R * SB);

  const int cta = blockIdx.x;
  const F32Tile T = f32_tile<TY>(a, cta);
  const BlockDev &B = a.blocks[T.b];
  const CavConst &C = a.cc[B.cav];
  const int li = threadIdx.x, lj = threadIdx.y, tid = lj * NTX + li;
  const F32QCol c = f32q_column(B, T, li, lj);
  const CUtensorMap *mapp = a.maps + 2 * (2 * T.b + a.parity), *mapo = mapp + 1;

  if (tid == 0) {
    for (int s = 0; s < R; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mapp) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mapo) : "memory");
  }
  __syncthreads();
  int issued = 0;
  // plane pl of the tile: the pressure box (arrays 0, 1; rows from node
  // j0-2) and the other box (arrays 2 .. 6; rows from node j0-1), one barrier
  auto issue = [&](int pl) {
    if (pl == a.withhold_plane) return;  // the timeout test: this plane never arrives
    const int s = pl % R;
    const int z = T.zbase + pl;
    mbar_expect_tx(&bars[s], f32_tx_bytes(TY));
    tma_load_4d(ring + s * SF, mapp, &bars[s], T.x0, T.y0, z, 0);
    tma_load_4d(ring + s * SF + PF, mapo, &bars[s], T.x0, T.y0 + 1, z, kF32NP);
  };
  if (tid == 0) {
    if (a.ghosts_late && f32_reads_ghosts<TY>(B, T)) {
      // the boxes reach a ghost layer, which the previous step's finalise
      // launch (this launch's programmatic predecessor, if any) writes
      asm volatile("griddepcontrol.wait;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    for (; issued < min(R, T.nplanes); ++issued) issue(issued);
  }
  auto wait_plane = [&](int pl) { return mbar_wait_bounded(&bars[pl % R], (uint32_t)((pl / R) & 1), a.wait_cycles); };
  auto slot = [&](int pl) { return ring + (pl % R) * SF; };

  const long long fs = B.fstride, plane = B.plane;
  const int nz = B.nz;
  // i is odd, so the pair starts on an 8-byte boundary of the row
  float *__restrict__ out = (float *)B.base[a.parity ^ 1] + node_index<float>(B, min(c.i, B.nx), min(c.j, B.ny), T.k0);

  bool bad = false;
  F32QAcc acc;
  f32q_clear(acc);
  for (int pl = 0; pl < 4; ++pl) {
    if (!bad && !wait_plane(pl)) bad = true;
    if (!bad) f32q_prologue_plane<NT, TY>(pl, slot(pl), T, c, tid, acc);
  }
  bad = __syncthreads_or(bad);
  // a programmatic dependent of the previous step's finalise: only now are its
  // dt, centre shift and reads of the partials complete (nothing global was
  // read from the state it writes, nor written, before this point)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const F32K<float2> K = f32_consts<float2>(C, a.cs[B.cav]);
  const F32K<float> K1 = f32_consts<float>(C, a.cs[B.cav]);
  if (!bad && tid == 0) {
    // the slots of planes 0 and 1 are free again
    for (; issued < min(R + 2, T.nplanes); ++issued) issue(issued);
  }

  for (int k = T.k0; k <= T.k1 && !bad; ++k) {
    const int pk = k - T.k0 + 2;  // plane index of k
    if (!wait_plane(pk + 2)) bad = true;
    if (!bad) {
      if (T.fix) fix_plane_walls<NT, TY>(slot(pk + 2), tid, T);
      if (c.act0)
        f32q_pair<TY>(slot(pk), slot(pk + 1), slot(pk + 2), K, K1, k, nz, T.wzl, T.wzh, a.local_dt, out, fs, c.colp,
                      c.col, c.wofs, c.act1, c.nus_warp, acc);
      out += plane;
    }
    bad = __syncthreads_or(bad);
    if (!bad && tid == 0 && issued < T.nplanes) {
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
  f32q_finish<NT>(a.partials, T.slot, tid, T, c, acc);
}

// Spectral-radius partials of the current state (no update), with the step
// kernel's tiling so that the finalise reduction reads the same layout.
template <class S, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) k_spectral(StepArgs a) {
  constexpr int NT = TX * TY;
  const TileRef R = f32_tile_ref(a.blocks, a.nblocks, a.ncoarse, blockIdx.x);
  const BlockDev &B = a.blocks[R.b];
  const CavConst &C = a.cc[B.cav];
  const int i = R.tx * TX + threadIdx.x + 1, j = R.ty * TY + threadIdx.y + 1;
  const int k0 = R.k0, k1 = R.k1;
  static_assert(std::is_same<S, float>::value, "the FP64 form refreshes its spectral radius in k_step_f64");
  // the FP32 bound the FP32-mixed step uses for every later dt
  const F32K<float> K = f32_spectral_consts(C);
  double smax = 0.0;
  if (i <= B.nx && j <= B.ny) {
    const S *q = (const S *)B.base[a.parity];
    const long long fs = B.fstride;
    constexpr int NP = Store<S>::NP;
    for (int k = k0; k <= k1; ++k) {
      const long long o = node_index<S>(B, i, j, k);
      smax = fmax(smax, (double)f32_spectral_exact(K, q[NP * fs + o], q[(NP + 1) * fs + o], q[(NP + 2) * fs + o]));
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
    a.partials[(long long)R.slot * kPartStride + tid] = acc;
  }
}

}  // namespace bdc
