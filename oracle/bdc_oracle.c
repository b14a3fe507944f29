/*
 * FP64 CPU oracle for one explicit time step of the artificial-compressibility
 * Boussinesq buoyancy-driven-cavity (BDC) solver of Xue & Roy (arXiv 2006.02602).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code with the CUDA path (paper_2006_02602_gb300/csrc) and neither side
 * includes or links the other.
 *
 * Plain triple loops, FP64, built with -ffp-contract=off (no FMA contraction),
 * every expression written in the paper's notation:
 *
 *   Eq. 1  (1/beta^2) dp/dt + rho dV_i/dx_i = eps_i d^4p/dx_i^4
 *   Eq. 2  dV_j/dt + V_i dV_j/dx_i = -(1/rho) dp/dx_j + nu d^2V_j/dx_i^2 + sigma (T - T_inf) g_j
 *   Eq. 3  dT/dt + V_i dT/dx_i = alpha d^2T/dx_i^2
 *
 * Section 2: first-order explicit Euler in (pseudo) time, second-order central
 * differences for every derivative, fourth-difference pressure dissipation on
 * the continuity equation only; pressure extrapolated to wall ghosts by a
 * one-sided second-order formula, temperature likewise at the adiabatic walls,
 * pressure rescaled at the cavity centre every iteration.
 * Section 3.1 / Fig. 1: stencil width 5 for p, 3 for u, v, w, T (star, no
 * diagonals); i fastest, k slowest.
 * Section 4.5, Listings 1-2 and "Optimized V3": ghost faces are packed into
 * contiguous buffers, p at depth 2, u, v, w, T at depth 1, on every cut face.
 *
 * Readings of points the paper leaves open:
 *  - thermal scaling: rho = 1, alpha = 1, nu = Pr, g*sigma = Ra*Pr, unit cube;
 *  - the dissipation acts with the damping sign (Eq. 1 read as
 *    dp/dt = -beta^2 (rho div V + sum_d eps_d delta_d^4 p / h_d^4));
 *  - beta^2 = max(|V|^2, kappa u_ref^2);
 *  - eps_d = c4 lambda_d h_d^3 / beta^2 with
 *    lambda_d = (|V_d| + sqrt(V_d^2 + 4 beta^2)) / 2;
 *  - dt = cfl / max over interior of
 *    [ sum_d lambda_d / h_d + 2 max(nu, alpha) sum_d 1/h_d^2 ];
 *  - vertex grid: n interior nodes per axis, walls are nodes 0 and n+1,
 *    h = 1/(n+1), one extra pressure ghost beyond each wall;
 *  - wall p:  p_w = 2 p_1 - p_2, ghost p_g = 2 p_w - p_1;
 *    adiabatic wall T: T_w = (4 T_1 - T_2) / 3; isothermal x walls;
 *    no-slip u = v = w = 0 on every wall;
 *  - centre rescale: subtract the mean of the 2^m nodes nearest the centre
 *    (m = number of even n_d), summed in lexicographic (k, j, i) order;
 *  - buoyancy +Ra Pr (T - T_inf) along the "up" axis (gravity_axis).
 * parity unpinned against the paper's own numbers: the paper prints no field
 * values, residuals or Nusselt numbers; every pin is a closed form, an
 * invariant or a brute-force comparison (tests/test_oracle_*.py).
 *
 * Array layout (one block): q[f][k+1][j+1][i+1], f = p,u,v,w,T, local node
 * index i in [-1, nx+2] (0 and nx+1 are wall or cut-face ghost nodes).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NF 5
enum { FP = 0, FU = 1, FV = 2, FW = 3, FT = 4 };

typedef struct {
  double Ra, Pr;        /* Rayleigh and Prandtl numbers */
  double cfl;           /* Courant number of the explicit step */
  double kappa;         /* beta^2 floor factor */
  double c4;            /* fourth-difference dissipation coefficient */
  double u_ref;         /* user reference velocity (Section 2) */
  double t_inf;         /* buoyancy reference temperature */
  double t_hot, t_cold; /* nominal isothermal wall temperatures */
  int gravity_axis;     /* 1 = y, 2 = z: buoyancy acts along +axis */
} orc_params;

typedef struct {
  int nx, ny, nz;    /* interior nodes of this block */
  int ox, oy, oz;    /* global node index = o + local node index */
  int gnx, gny, gnz; /* interior nodes of the whole cavity */
  int wall[6];       /* face -x,+x,-y,+y,-z,+z lies on a cavity wall */
} orc_block;

static size_t ex_(const orc_block *b) { return (size_t)b->nx + 4; }
static size_t ey_(const orc_block *b) { return (size_t)b->ny + 4; }
static size_t ez_(const orc_block *b) { return (size_t)b->nz + 4; }

size_t orc_block_points(const orc_block *b) { return ex_(b) * ey_(b) * ez_(b); }

/* linear index of node (i,j,k) of field f */
static size_t at(const orc_block *b, int f, int i, int j, int k) {
  return (size_t)(i + 1) +
         ex_(b) * ((size_t)(j + 1) + ey_(b) * ((size_t)(k + 1) + ez_(b) * (size_t)f));
}

static void spacings(const orc_block *b, double h[3]) {
  h[0] = 1.0 / (double)(b->gnx + 1);
  h[1] = 1.0 / (double)(b->gny + 1);
  h[2] = 1.0 / (double)(b->gnz + 1);
}

/* ------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea & Flood 2014; Vigna's public-domain C form):
 * the value returned for state x is the generator's next output after its
 * state has been advanced from x by the golden-ratio increment. */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* uniform in [0,1) from the top 53 bits */
static double uniform01(uint64_t key) {
  return (double)(orc_splitmix64(key) >> 11) * (1.0 / 9007199254740992.0);
}

/* Initial state (configuration text: u = v = w = p = 0, T linear in x plus
 * uniform noise of amplitude a).  Noise draw for global interior node
 * (I,J,K), 1-based: U = uniform01(seed * 2^40 + gidx), gidx = (I-1) +
 * gnx ((J-1) + gny (K-1)); T = t_hot + (t_cold - t_hot) x + a (2U - 1).
 * Walls and ghosts are left at zero; the caller applies orc_bc next. */
void orc_init(const orc_params *P, const orc_block *b, double *q, uint64_t seed,
              double noise_amp) {
  double h[3];
  spacings(b, h);
  memset(q, 0, sizeof(double) * NF * orc_block_points(b));
  for (int k = 1; k <= b->nz; ++k)
    for (int j = 1; j <= b->ny; ++j)
      for (int i = 1; i <= b->nx; ++i) {
        const int I = b->ox + i, J = b->oy + j, K = b->oz + k;
        const uint64_t gidx = (uint64_t)(I - 1) +
                              (uint64_t)b->gnx * ((uint64_t)(J - 1) + (uint64_t)b->gny * (uint64_t)(K - 1));
        const double U = uniform01(seed * (1ULL << 40) + gidx);
        const double x = (double)I * h[0];
        q[at(b, FT, i, j, k)] = P->t_hot + (P->t_cold - P->t_hot) * x + noise_amp * (2.0 * U - 1.0);
      }
}

/* ------------------------------------------------------------------ */
/* Time derivatives dq/dt of Eqs. 1-3 at every interior node of the block.
 * dqdt layout: [f][k-1][j-1][i-1] over the block interior.  Reads the
 * 13-point pressure star and the 7-point star of u, v, w, T (Fig. 1). */
void orc_rates(const orc_params *P, const orc_block *b, const double *q, double *dqdt) {
  double h[3];
  spacings(b, h);
  const double rho = 1.0, nu = P->Pr, alpha = 1.0, gsigma = P->Ra * P->Pr;
  const double beta2_floor = P->kappa * P->u_ref * P->u_ref;
  const size_t nint = (size_t)b->nx * b->ny * b->nz;
  const int nx = b->nx, ny = b->ny, nz = b->nz;
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= nz; ++k)
    for (int j = 1; j <= ny; ++j)
      for (int i = 1; i <= nx; ++i) {
        /* unit offsets along x, y, z */
        const int di[3] = {1, 0, 0}, dj[3] = {0, 1, 0}, dk[3] = {0, 0, 1};
        double V[3];
        V[0] = q[at(b, FU, i, j, k)];
        V[1] = q[at(b, FV, i, j, k)];
        V[2] = q[at(b, FW, i, j, k)];
        const double p0 = q[at(b, FP, i, j, k)];
        const double T0 = q[at(b, FT, i, j, k)];

        /* local artificial compressibility (Section 2: local velocity
         * magnitude with a user reference velocity) */
        double beta2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
        if (beta2 < beta2_floor) beta2 = beta2_floor;

        /* Eq. 1: continuity residual with fourth-difference dissipation */
        double divV = 0.0, dissip = 0.0;
        for (int d = 0; d < 3; ++d) {
          const double Vp = q[at(b, FU + d, i + di[d], j + dj[d], k + dk[d])];
          const double Vm = q[at(b, FU + d, i - di[d], j - dj[d], k - dk[d])];
          divV += (Vp - Vm) / (2.0 * h[d]);

          const double pp2 = q[at(b, FP, i + 2 * di[d], j + 2 * dj[d], k + 2 * dk[d])];
          const double pp1 = q[at(b, FP, i + di[d], j + dj[d], k + dk[d])];
          const double pm1 = q[at(b, FP, i - di[d], j - dj[d], k - dk[d])];
          const double pm2 = q[at(b, FP, i - 2 * di[d], j - 2 * dj[d], k - 2 * dk[d])];
          const double delta4 = pp2 - 4.0 * pp1 + 6.0 * p0 - 4.0 * pm1 + pm2;
          const double lambda = 0.5 * (fabs(V[d]) + sqrt(V[d] * V[d] + 4.0 * beta2));
          const double eps = P->c4 * lambda * h[d] * h[d] * h[d] / beta2;
          dissip += eps * delta4 / (h[d] * h[d] * h[d] * h[d]);
        }
        const double Rp = rho * divV + dissip;
        const size_t o = (size_t)(i - 1) + (size_t)nx * ((size_t)(j - 1) + (size_t)ny * (size_t)(k - 1));
        dqdt[FP * nint + o] = -beta2 * Rp;

        /* Eq. 2: momentum, component c */
        for (int c = 0; c < 3; ++c) {
          const double Vc = V[c];
          double conv = 0.0, lap = 0.0;
          for (int d = 0; d < 3; ++d) {
            const double qp = q[at(b, FU + c, i + di[d], j + dj[d], k + dk[d])];
            const double qm = q[at(b, FU + c, i - di[d], j - dj[d], k - dk[d])];
            conv += V[d] * (qp - qm) / (2.0 * h[d]);
            lap += (qp - 2.0 * Vc + qm) / (h[d] * h[d]);
          }
          const double pp = q[at(b, FP, i + di[c], j + dj[c], k + dk[c])];
          const double pm = q[at(b, FP, i - di[c], j - dj[c], k - dk[c])];
          const double gradp = (pp - pm) / (2.0 * h[c]);
          const double buoy = (c == P->gravity_axis) ? gsigma * (T0 - P->t_inf) : 0.0;
          dqdt[(size_t)(FU + c) * nint + o] = -conv - gradp / rho + nu * lap + buoy;
        }

        /* Eq. 3: energy */
        {
          double conv = 0.0, lap = 0.0;
          for (int d = 0; d < 3; ++d) {
            const double qp = q[at(b, FT, i + di[d], j + dj[d], k + dk[d])];
            const double qm = q[at(b, FT, i - di[d], j - dj[d], k - dk[d])];
            conv += V[d] * (qp - qm) / (2.0 * h[d]);
            lap += (qp - 2.0 * T0 + qm) / (h[d] * h[d]);
          }
          dqdt[FT * nint + o] = -conv + alpha * lap;
        }
      }
}

/* Spectral-radius bound of the explicit step at node (i, j, k): the sum over
 * axes of the acoustic wave speeds lambda_d / h_d plus the diffusive term
 * 2 max(nu, alpha) sum 1/h_d^2 (Section 2, the stable dt). */
static double node_spectral(const orc_params *P, const orc_block *b, const double *q, const double h[3], int i, int j,
                            int k) {
  const double nu = P->Pr, alpha = 1.0;
  const double beta2_floor = P->kappa * P->u_ref * P->u_ref;
  const double dmax = nu > alpha ? nu : alpha;
  const double diff = 2.0 * dmax * (1.0 / (h[0] * h[0]) + 1.0 / (h[1] * h[1]) + 1.0 / (h[2] * h[2]));
  double V[3];
  V[0] = q[at(b, FU, i, j, k)];
  V[1] = q[at(b, FV, i, j, k)];
  V[2] = q[at(b, FW, i, j, k)];
  double beta2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
  if (beta2 < beta2_floor) beta2 = beta2_floor;
  double s = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double lambda = 0.5 * (fabs(V[d]) + sqrt(V[d] * V[d] + 4.0 * beta2));
    s += lambda / h[d];
  }
  return s + diff;
}

/* Largest spectral-radius bound over the block interior (the denominator of
 * the stable explicit dt); max is exact, so the result does not depend on
 * the loop order. */
double orc_spectral_max(const orc_params *P, const orc_block *b, const double *q) {
  double h[3];
  spacings(b, h);
  double smax = 0.0;
  const int nx = b->nx, ny = b->ny, nz = b->nz;
#pragma omp parallel for schedule(static) reduction(max : smax)
  for (int k = 1; k <= nz; ++k)
    for (int j = 1; j <= ny; ++j)
      for (int i = 1; i <= nx; ++i) {
        const double s = node_spectral(P, b, q, h, i, j, k);
        if (s > smax) smax = s;
      }
  return smax;
}

/* Explicit Euler update q <- q + dt dq/dt on the interior.  sumsq[f] gets the
 * sum over the block interior of (dq_f/dt)^2, accumulated plane by plane and
 * then over planes in increasing k, so the result is independent of the
 * thread count. */
void orc_update(const orc_block *b, double *q, const double *dqdt, double dt, double *sumsq) {
  const int nx = b->nx, ny = b->ny, nz = b->nz;
  const size_t nint = (size_t)nx * ny * nz;
  double *plane = (double *)calloc((size_t)nz * NF, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= nz; ++k)
    for (int f = 0; f < NF; ++f) {
      double s = 0.0;
      for (int j = 1; j <= ny; ++j)
        for (int i = 1; i <= nx; ++i) {
          const size_t o = (size_t)(i - 1) + (size_t)nx * ((size_t)(j - 1) + (size_t)ny * (size_t)(k - 1));
          const double r = dqdt[(size_t)f * nint + o];
          q[at(b, f, i, j, k)] = q[at(b, f, i, j, k)] + dt * r;
          s += r * r;
        }
      plane[(size_t)(k - 1) * NF + f] = s;
    }
  for (int f = 0; f < NF; ++f) {
    double s = 0.0;
    for (int k = 0; k < nz; ++k) s += plane[(size_t)k * NF + f];
    sumsq[f] = s;
  }
  free(plane);
}

/* Local time stepping (the iteration in pseudo time of Section 3.1, each node
 * at its own stable step): q <- q + dt_n dq/dt with dt_n = cfl / S_n, S_n the
 * spectral bound of node n in the state before the update (all dt_n are
 * taken before any node changes).  sumsq as in orc_update. */
void orc_update_local(const orc_params *P, const orc_block *b, double *q, const double *dqdt, double *sumsq) {
  const int nx = b->nx, ny = b->ny, nz = b->nz;
  const size_t nint = (size_t)nx * ny * nz;
  double h[3];
  spacings(b, h);
  double *dtl = (double *)malloc(nint * sizeof(double));
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= nz; ++k)
    for (int j = 1; j <= ny; ++j)
      for (int i = 1; i <= nx; ++i) {
        const size_t o = (size_t)(i - 1) + (size_t)nx * ((size_t)(j - 1) + (size_t)ny * (size_t)(k - 1));
        dtl[o] = P->cfl / node_spectral(P, b, q, h, i, j, k);
      }
  double *plane = (double *)calloc((size_t)nz * NF, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= nz; ++k)
    for (int f = 0; f < NF; ++f) {
      double s = 0.0;
      for (int j = 1; j <= ny; ++j)
        for (int i = 1; i <= nx; ++i) {
          const size_t o = (size_t)(i - 1) + (size_t)nx * ((size_t)(j - 1) + (size_t)ny * (size_t)(k - 1));
          const double r = dqdt[(size_t)f * nint + o];
          q[at(b, f, i, j, k)] = q[at(b, f, i, j, k)] + dtl[o] * r;
          s += r * r;
        }
      plane[(size_t)(k - 1) * NF + f] = s;
    }
  for (int f = 0; f < NF; ++f) {
    double s = 0.0;
    for (int k = 0; k < nz; ++k) s += plane[(size_t)k * NF + f];
    sumsq[f] = s;
  }
  free(plane);
  free(dtl);
}

/* Section 2: pressure rescaled at the centre -- subtract c from interior p. */
void orc_shift_pressure(const orc_block *b, double *q, double c) {
  for (int k = 1; k <= b->nz; ++k)
    for (int j = 1; j <= b->ny; ++j)
      for (int i = 1; i <= b->nx; ++i) q[at(b, FP, i, j, k)] -= c;
}

/* Wall boundary conditions (Section 2) on the faces of this block that lie
 * on a cavity wall, over the face's interior node range.  Wall node w,
 * first two interior nodes 1, 2, pressure ghost g beyond the wall:
 *   u = v = w = 0 (no slip);
 *   p_w = 2 p_1 - p_2, p_g = 2 p_w - p_1 (one-sided second order);
 *   T_w = (4 T_1 - T_2) / 3 on adiabatic walls, T_w = wall temperature on
 *   the isothermal x walls (t_hot_w at x = 0, t_cold_w at x = 1, each
 *   gny*gnz values indexed (J-1) + gny (K-1) by global node index). */
void orc_bc(const orc_block *b, double *q, const double *t_hot_w, const double *t_cold_w) {
  for (int face = 0; face < 6; ++face) {
    if (!b->wall[face]) continue;
    const int axis = face / 2, high = face % 2;
    const int n[3] = {b->nx, b->ny, b->nz};
    const int a1 = axis == 0 ? 1 : 0;          /* first face axis  */
    const int a2 = axis == 2 ? 1 : 2;          /* second face axis */
    const int w = high ? n[axis] + 1 : 0;      /* wall node */
    const int s = high ? -1 : 1;               /* step into the interior */
    for (int c2 = 1; c2 <= n[a2]; ++c2)
      for (int c1 = 1; c1 <= n[a1]; ++c1) {
        int iw[3], i1[3], i2[3], ig[3];
        iw[axis] = w; i1[axis] = w + s; i2[axis] = w + 2 * s; ig[axis] = w - s;
        iw[a1] = i1[a1] = i2[a1] = ig[a1] = c1;
        iw[a2] = i1[a2] = i2[a2] = ig[a2] = c2;
        const size_t W = at(b, 0, iw[0], iw[1], iw[2]);
        const size_t N1 = at(b, 0, i1[0], i1[1], i1[2]);
        const size_t N2 = at(b, 0, i2[0], i2[1], i2[2]);
        const size_t G = at(b, 0, ig[0], ig[1], ig[2]);
        const size_t fs = orc_block_points(b); /* field stride */
        q[FU * fs + W] = 0.0;
        q[FV * fs + W] = 0.0;
        q[FW * fs + W] = 0.0;
        const double pw = 2.0 * q[FP * fs + N1] - q[FP * fs + N2];
        q[FP * fs + W] = pw;
        q[FP * fs + G] = 2.0 * pw - q[FP * fs + N1];
        if (axis == 0) {
          const int J = b->oy + iw[1], K = b->oz + iw[2];
          const size_t widx = (size_t)(J - 1) + (size_t)b->gny * (size_t)(K - 1);
          q[FT * fs + W] = high ? t_cold_w[widx] : t_hot_w[widx];
        } else {
          q[FT * fs + W] = (4.0 * q[FT * fs + N1] - q[FT * fs + N2]) / 3.0;
        }
      }
  }
}

/* Hot- and cold-wall Nusselt sums of this block: sum over its x-wall face
 * nodes of the one-sided second-order wall heat flux -dT/dx divided by
 * (t_hot - t_cold).  The caller divides by gny*gnz. */
void orc_nusselt_sums(const orc_params *P, const orc_block *b, const double *q, double *hot,
                      double *cold) {
  double h[3];
  spacings(b, h);
  const double dT = P->t_hot - P->t_cold;
  double sh = 0.0, sc = 0.0;
  for (int k = 1; k <= b->nz; ++k)
    for (int j = 1; j <= b->ny; ++j) {
      if (b->wall[0]) {
        const double T0 = q[at(b, FT, 0, j, k)], T1 = q[at(b, FT, 1, j, k)], T2 = q[at(b, FT, 2, j, k)];
        sh += (3.0 * T0 - 4.0 * T1 + T2) / (2.0 * h[0]) / dT;
      }
      if (b->wall[1]) {
        const int n = b->nx;
        const double T0 = q[at(b, FT, n + 1, j, k)], T1 = q[at(b, FT, n, j, k)], T2 = q[at(b, FT, n - 1, j, k)];
        sc += (-3.0 * T0 + 4.0 * T1 - T2) / (2.0 * h[0]) / dT;
      }
    }
  *hot = sh;
  *cold = sc;
}

/* ------------------------------------------------------------------ */
/* Ghost-face exchange buffers (Section 4.5, Listings 1-2, Optimized V3).
 * Face f: axis a = f/2, low (f even) or high (f odd) side.  The two face
 * axes are the remaining axes in increasing order, b (faster) and c.
 * Buffer: pressure first, depth fastest, then b, then c:
 *     buf[(ic * nb + ib) * 2 + d]                      d = 0, 1
 * then u, v, w, T at depth 1, b fastest, then c, then the variable:
 *     buf[2 nb nc + v nb nc + ic nb + ib]              v = 0..3
 * Depth d counts layers in increasing index order.  Packed layers: p from
 * local layers {1, 2} (low face) or {n-1, n} (high face); u, v, w, T from
 * layer 1 (low) or n (high).  Length 6 nb nc. */
static void face_axes(int face, int *a, int *bb, int *cc) {
  *a = face / 2;
  *bb = *a == 0 ? 1 : 0;
  *cc = *a == 2 ? 1 : 2;
}

size_t orc_face_len(const orc_block *b, int face) {
  int a, bb, cc;
  face_axes(face, &a, &bb, &cc);
  const int n[3] = {b->nx, b->ny, b->nz};
  return (size_t)6 * n[bb] * n[cc];
}

void orc_pack(const orc_block *b, const double *q, int face, double *buf) {
  int a, bb, cc;
  face_axes(face, &a, &bb, &cc);
  const int n[3] = {b->nx, b->ny, b->nz};
  const int nb = n[bb], nc = n[cc];
  const int high = face % 2;
  const int p_first = high ? n[a] - 1 : 1; /* first packed pressure layer */
  const int v_layer = high ? n[a] : 1;     /* packed layer of u, v, w, T */
  const size_t plane = (size_t)nb * nc;
  for (int ic = 0; ic < nc; ++ic)
    for (int ib = 0; ib < nb; ++ib) {
      int idx[3];
      idx[bb] = ib + 1;
      idx[cc] = ic + 1;
      for (int d = 0; d < 2; ++d) {
        idx[a] = p_first + d;
        buf[((size_t)ic * nb + ib) * 2 + d] = q[at(b, FP, idx[0], idx[1], idx[2])];
      }
      idx[a] = v_layer;
      for (int v = 0; v < 4; ++v)
        buf[2 * plane + (size_t)v * plane + (size_t)ic * nb + ib] = q[at(b, FU + v, idx[0], idx[1], idx[2])];
    }
}

/* Unpack a neighbour's buffer into the ghost layers of this block's face
 * `face`: high face -> layers n+1, n+2 (p) and n+1 (u, v, w, T); low face ->
 * layers -1, 0 (p) and 0 (u, v, w, T). */
void orc_unpack(const orc_block *b, double *q, int face, const double *buf) {
  int a, bb, cc;
  face_axes(face, &a, &bb, &cc);
  const int n[3] = {b->nx, b->ny, b->nz};
  const int nb = n[bb], nc = n[cc];
  const int high = face % 2;
  const int p_first = high ? n[a] + 1 : -1;
  const int v_layer = high ? n[a] + 1 : 0;
  const size_t plane = (size_t)nb * nc;
  for (int ic = 0; ic < nc; ++ic)
    for (int ib = 0; ib < nb; ++ib) {
      int idx[3];
      idx[bb] = ib + 1;
      idx[cc] = ic + 1;
      for (int d = 0; d < 2; ++d) {
        idx[a] = p_first + d;
        q[at(b, FP, idx[0], idx[1], idx[2])] = buf[((size_t)ic * nb + ib) * 2 + d];
      }
      idx[a] = v_layer;
      for (int v = 0; v < 4; ++v)
        q[at(b, FU + v, idx[0], idx[1], idx[2])] = buf[2 * plane + (size_t)v * plane + (size_t)ic * nb + ib];
    }
}

/* ------------------------------------------------------------------ */
/* Discrete adjoint of the rates (reverse of orc_rates, node by node).
 * Given rbar[f][k-1][j-1][i-1] (adjoint of dq/dt at every interior node),
 * accumulate into qbar (same layout as q, walls and ghosts included) the
 * transposed Jacobian product, and into pbar[0] the adjoint of g*sigma
 * (= Ra Pr), into pbar[1] the adjoint of the beta^2 floor kappa u_ref^2.
 * Subgradients at the kinks: |x|' = sign(x) with sign(0) = 0; the max in
 * beta^2 follows the branch taken.  Sequential: the scatter to the stencil
 * inputs has no write conflicts. */
void orc_rates_vjp(const orc_params *P, const orc_block *b, const double *q, const double *rbar, double *qbar,
                   double *pbar) {
  double h[3];
  spacings(b, h);
  const double nu = P->Pr, alpha = 1.0;
  const double beta2_floor = P->kappa * P->u_ref * P->u_ref;
  const size_t nint = (size_t)b->nx * b->ny * b->nz;
  const int di[3] = {1, 0, 0}, dj[3] = {0, 1, 0}, dk[3] = {0, 0, 1};
  double gsbar = 0.0, floorbar = 0.0;
  for (int k = 1; k <= b->nz; ++k)
    for (int j = 1; j <= b->ny; ++j)
      for (int i = 1; i <= b->nx; ++i) {
        const size_t o = (size_t)(i - 1) + (size_t)b->nx * ((size_t)(j - 1) + (size_t)b->ny * (size_t)(k - 1));
        const double rp = rbar[FP * nint + o], rT = rbar[FT * nint + o];
        const double rV[3] = {rbar[FU * nint + o], rbar[FV * nint + o], rbar[FW * nint + o]};
        double V[3];
        for (int d = 0; d < 3; ++d) V[d] = q[at(b, FU + d, i, j, k)];
        const double p0 = q[at(b, FP, i, j, k)];
        const double T0 = q[at(b, FT, i, j, k)];
        double Vbar[3] = {0.0, 0.0, 0.0};
        /* forward intermediates */
        double beta2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
        const int floored = beta2 < beta2_floor;
        if (floored) beta2 = beta2_floor;
        double divV = 0.0, dissip = 0.0, delta4[3], lambda[3], sq[3], eps[3];
        for (int d = 0; d < 3; ++d) {
          const double Vp = q[at(b, FU + d, i + di[d], j + dj[d], k + dk[d])];
          const double Vm = q[at(b, FU + d, i - di[d], j - dj[d], k - dk[d])];
          divV += (Vp - Vm) / (2.0 * h[d]);
          const double pp2 = q[at(b, FP, i + 2 * di[d], j + 2 * dj[d], k + 2 * dk[d])];
          const double pp1 = q[at(b, FP, i + di[d], j + dj[d], k + dk[d])];
          const double pm1 = q[at(b, FP, i - di[d], j - dj[d], k - dk[d])];
          const double pm2 = q[at(b, FP, i - 2 * di[d], j - 2 * dj[d], k - 2 * dk[d])];
          delta4[d] = pp2 - 4.0 * pp1 + 6.0 * p0 - 4.0 * pm1 + pm2;
          sq[d] = sqrt(V[d] * V[d] + 4.0 * beta2);
          lambda[d] = 0.5 * (fabs(V[d]) + sq[d]);
          eps[d] = P->c4 * lambda[d] * h[d] * h[d] * h[d] / beta2;
          dissip += eps[d] * delta4[d] / (h[d] * h[d] * h[d] * h[d]);
        }
        const double Rp = divV + dissip;
        double beta2bar = 0.0;

        /* energy: dT/dt = -sum V_d dT/dx_d + alpha lap T */
        for (int d = 0; d < 3; ++d) {
          const double Tp = q[at(b, FT, i + di[d], j + dj[d], k + dk[d])];
          const double Tm = q[at(b, FT, i - di[d], j - dj[d], k - dk[d])];
          const double cbar = -rT, lbar = alpha * rT;
          qbar[at(b, FT, i + di[d], j + dj[d], k + dk[d])] += cbar * V[d] / (2.0 * h[d]) + lbar / (h[d] * h[d]);
          qbar[at(b, FT, i - di[d], j - dj[d], k - dk[d])] += -cbar * V[d] / (2.0 * h[d]) + lbar / (h[d] * h[d]);
          qbar[at(b, FT, i, j, k)] += -2.0 * lbar / (h[d] * h[d]);
          Vbar[d] += cbar * (Tp - Tm) / (2.0 * h[d]);
        }
        /* momentum component c */
        for (int c = 0; c < 3; ++c) {
          const double cbar = -rV[c], lbar = nu * rV[c];
          for (int d = 0; d < 3; ++d) {
            const double qp = q[at(b, FU + c, i + di[d], j + dj[d], k + dk[d])];
            const double qm = q[at(b, FU + c, i - di[d], j - dj[d], k - dk[d])];
            qbar[at(b, FU + c, i + di[d], j + dj[d], k + dk[d])] += cbar * V[d] / (2.0 * h[d]) + lbar / (h[d] * h[d]);
            qbar[at(b, FU + c, i - di[d], j - dj[d], k - dk[d])] += -cbar * V[d] / (2.0 * h[d]) + lbar / (h[d] * h[d]);
            Vbar[c] += -2.0 * lbar / (h[d] * h[d]);
            Vbar[d] += cbar * (qp - qm) / (2.0 * h[d]);
          }
          qbar[at(b, FP, i + di[c], j + dj[c], k + dk[c])] += -rV[c] / (2.0 * h[c]);
          qbar[at(b, FP, i - di[c], j - dj[c], k - dk[c])] += rV[c] / (2.0 * h[c]);
          if (c == P->gravity_axis) {
            qbar[at(b, FT, i, j, k)] += P->Ra * P->Pr * rV[c];
            gsbar += (T0 - P->t_inf) * rV[c];
          }
        }
        /* continuity: dp/dt = -beta^2 (divV + sum_d eps_d delta4_d / h_d^4) */
        beta2bar += -Rp * rp;
        const double Rpbar = -beta2 * rp;
        for (int d = 0; d < 3; ++d) {
          qbar[at(b, FU + d, i + di[d], j + dj[d], k + dk[d])] += Rpbar / (2.0 * h[d]);
          qbar[at(b, FU + d, i - di[d], j - dj[d], k - dk[d])] += -Rpbar / (2.0 * h[d]);
          const double h4 = h[d] * h[d] * h[d] * h[d];
          const double epsbar = Rpbar * delta4[d] / h4;
          const double d4bar = Rpbar * eps[d] / h4;
          qbar[at(b, FP, i + 2 * di[d], j + 2 * dj[d], k + 2 * dk[d])] += d4bar;
          qbar[at(b, FP, i + di[d], j + dj[d], k + dk[d])] += -4.0 * d4bar;
          qbar[at(b, FP, i, j, k)] += 6.0 * d4bar;
          qbar[at(b, FP, i - di[d], j - dj[d], k - dk[d])] += -4.0 * d4bar;
          qbar[at(b, FP, i - 2 * di[d], j - 2 * dj[d], k - 2 * dk[d])] += d4bar;
          const double h3 = h[d] * h[d] * h[d];
          const double lambdabar = epsbar * P->c4 * h3 / beta2;
          beta2bar += -epsbar * P->c4 * lambda[d] * h3 / (beta2 * beta2);
          const double sgn = V[d] > 0.0 ? 1.0 : (V[d] < 0.0 ? -1.0 : 0.0);
          Vbar[d] += lambdabar * 0.5 * (sgn + V[d] / sq[d]);
          beta2bar += lambdabar * 0.5 * (2.0 / sq[d]);
        }
        if (floored) {
          floorbar += beta2bar;
        } else {
          for (int d = 0; d < 3; ++d) Vbar[d] += beta2bar * 2.0 * V[d];
        }
        for (int d = 0; d < 3; ++d) qbar[at(b, FU + d, i, j, k)] += Vbar[d];
      }
  pbar[0] += gsbar;
  pbar[1] += floorbar;
}

/* Node (1-based interior i, j, k) where the spectral-radius bound is largest
 * (first in k, j, i order among equal values); returns the maximum. */
double orc_spectral_argmax(const orc_params *P, const orc_block *b, const double *q, int *idx) {
  double h[3];
  spacings(b, h);
  const double nu = P->Pr, alpha = 1.0;
  const double beta2_floor = P->kappa * P->u_ref * P->u_ref;
  const double dmax = nu > alpha ? nu : alpha;
  const double diff = 2.0 * dmax * (1.0 / (h[0] * h[0]) + 1.0 / (h[1] * h[1]) + 1.0 / (h[2] * h[2]));
  double smax = -1.0;
  for (int k = 1; k <= b->nz; ++k)
    for (int j = 1; j <= b->ny; ++j)
      for (int i = 1; i <= b->nx; ++i) {
        double V[3];
        V[0] = q[at(b, FU, i, j, k)];
        V[1] = q[at(b, FV, i, j, k)];
        V[2] = q[at(b, FW, i, j, k)];
        double beta2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
        if (beta2 < beta2_floor) beta2 = beta2_floor;
        double s = 0.0;
        for (int d = 0; d < 3; ++d) s += 0.5 * (fabs(V[d]) + sqrt(V[d] * V[d] + 4.0 * beta2)) / h[d];
        s += diff;
        if (s > smax) {
          smax = s;
          idx[0] = i; idx[1] = j; idx[2] = k;
        }
      }
  return smax;
}

/* Adjoint of the spectral-radius bound at node (i, j, k): qbar of u, v, w
 * there += sbar * d(bound)/dV, pbar[1] (beta^2 floor) += sbar * d/dfloor. */
void orc_spectral_vjp(const orc_params *P, const orc_block *b, const double *q, int i, int j, int k, double sbar,
                      double *qbar, double *pbar) {
  double h[3];
  spacings(b, h);
  const double beta2_floor = P->kappa * P->u_ref * P->u_ref;
  double V[3];
  for (int d = 0; d < 3; ++d) V[d] = q[at(b, FU + d, i, j, k)];
  double beta2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
  const int floored = beta2 < beta2_floor;
  if (floored) beta2 = beta2_floor;
  double beta2bar = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double sq = sqrt(V[d] * V[d] + 4.0 * beta2);
    const double lambdabar = sbar / h[d];
    const double sgn = V[d] > 0.0 ? 1.0 : (V[d] < 0.0 ? -1.0 : 0.0);
    qbar[at(b, FU + d, i, j, k)] += lambdabar * 0.5 * (sgn + V[d] / sq);
    beta2bar += lambdabar * 0.5 * (2.0 / sq);
  }
  if (floored) {
    pbar[1] += beta2bar;
  } else {
    for (int d = 0; d < 3; ++d) qbar[at(b, FU + d, i, j, k)] += beta2bar * 2.0 * V[d];
  }
}
