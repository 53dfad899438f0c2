/*
 * fmm_oracle.c -- plain, slow FP64 CPU oracle for the unigrid FMM Poisson
 * solve with isolated boundaries of Lee & Teyssier, "A Scalable Fast
 * Multipole Method Poisson Solver for the RAMSES code: I. Unigrid Algorithm".
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this library.  The product (CUDA) path
 * shares no code, header, table or helper with it.
 *
 * Every function states the passage of the paper it follows.  Conventions
 * (the places where the paper is silent or ambiguous are resolved as listed
 * in the repository's design notes, "readings Q1-Q13"):
 *
 *  - Cell units: cell (i,j,k) has centre (i+1/2, j+1/2, k+1/2); cell mass
 *    m = rho (the physical potential is G*dx^2 times the cell-unit one).
 *  - Arrays are [nz][ny][nx], x fastest.
 *  - Multi-indices alpha=(a,b,c), |alpha| <= p, canonical order: by total
 *    order n, then a descending, then b descending.
 *  - Moments M_alpha = sum m (x - c)^alpha           (Sec. 2.1, eq. multipole,
 *    taken about the FMM cell centre; the origin form of Sec. 2.1 followed by
 *    eq. M2M_general gives the same numbers, see oracle_upward_origin()).
 *  - M2L (Sec. 2.3, eq. M2L, written per multi-index):
 *        L_beta = sum_{|alpha| <= p-|beta|} (-1)^|alpha| / alpha!
 *                 * D_{alpha+beta}(R) * M_alpha,
 *    D_gamma = d^gamma g, g(R) = -1/|R|, R = c_target - c_source (reading Q1).
 *  - L2L (eq. L2L): L'_beta = sum_{gamma>=beta} a^(gamma-beta)/(gamma-beta)!
 *    * L_gamma, a = c_child - c_parent.
 *  - L2P: phi(x) = sum_beta L_beta (x-c)^beta / beta!.
 *  - Near field (eq. direct): g(r) = -1/|r|, g(0) = -1/dx (self cell kept).
 *  - Interaction list (Sec. 2.2): children of the parent's 3^3 neighbour
 *    cells that are not themselves neighbours (Chebyshev distance >= 2),
 *    clipped to the domain (isolated boundary).
 *  - Hierarchy (Sec. 2): finest FMM level has leaf boxes of b^3 cells; each
 *    coarser level halves the box count per axis (rounding up, the boxes
 *    past the domain carry no mass) until one box remains (level 0).
 *
 * Multipole and local truncation: |alpha| + |beta| <= p (symmetric, reading
 * Q2), so that the whole operator is symmetric.
 *
 * Mutation hooks (ORACLE_MUTANT=k) exist only so the test-suite can build
 * deliberately broken copies of this oracle and check that its pins catch
 * each mistake.  The default build (ORACLE_MUTANT undefined / 0) is the
 * oracle.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#define OR_MAXP 12
#define OR_MAXLEV 40

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */
/* ------------------------------------------------------------------------ */

static double or_ipow(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

static double or_fact(int k) {
  double r = 1.0;
  for (int i = 2; i <= k; ++i) r *= (double)i;
  return r;
}

static double or_binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  return or_fact(n) / (or_fact(k) * or_fact(n - k));
}

int oracle_ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

/* Canonical multi-index list for order p: writes 3*ncoef(p) ints. */
typedef struct {
  int p, nc;
  int mo, lo;            /* multipole / local order limits inside |alpha| + |beta| <= p (default p) */
  int mi[1000][3];       /* ncoef(12) = 455 < 1000 */
  int lut[OR_MAXP + 1][OR_MAXP + 1][OR_MAXP + 1];
} or_index;

static void or_index_init(or_index* ix, int p) {
  ix->p = p;
  ix->mo = ix->lo = p;
  int k = 0;
  for (int a = 0; a <= OR_MAXP; ++a)
    for (int b = 0; b <= OR_MAXP; ++b)
      for (int c = 0; c <= OR_MAXP; ++c) ix->lut[a][b][c] = -1;
  for (int n = 0; n <= p; ++n)
    for (int a = n; a >= 0; --a)
      for (int b = n - a; b >= 0; --b) {
        int c = n - a - b;
        ix->mi[k][0] = a;
        ix->mi[k][1] = b;
        ix->mi[k][2] = c;
        ix->lut[a][b][c] = k;
        ++k;
      }
  ix->nc = k;
}

int oracle_index(int p, int* out) {
  if (p < 0 || p > OR_MAXP) return -1;
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  for (int k = 0; k < ix->nc; ++k)
    for (int d = 0; d < 3; ++d) out[3 * k + d] = ix->mi[k][d];
  int nc = ix->nc;
  free(ix);
  return nc;
}

/* ------------------------------------------------------------------------ */
/* Derivative tensor D_gamma(R) = d^gamma (-1/|R|), |gamma| <= order.       */
/* Method: McMurchie-Davidson Hermite recursion for 1/r:                    */
/*   R^(n)_000   = (-1)^n (2n-1)!! / r^(2n+1)                               */
/*   R^(n)_{t+1,u,v} = t R^(n+1)_{t-1,u,v} + X R^(n+1)_{t,u,v}  (same in u,v)*/
/*   d^{tuv}(1/r) = R^(0)_{tuv}.                                            */
/* This is the "Green's function and its Taylor expansion" that Sec. 2.2    */
/* precomputes for the fixed interaction geometry; the oracle simply        */
/* evaluates it for every pair.                                             */
/* ------------------------------------------------------------------------ */

static void or_dtensor_ix(const or_index* ix, const double R[3], int order, double* D) {
  const int P1 = order + 1;
  const int sz = P1 * P1 * P1 * P1;
  double* H = (double*)malloc(sizeof(double) * (size_t)sz);
#define HI(n, t, u, v) ((((n) * P1 + (t)) * P1 + (u)) * P1 + (v))
  const double X = R[0], Y = R[1], Z = R[2];
  const double r2 = X * X + Y * Y + Z * Z;
  const double r = sqrt(r2);
  /* base: (-1)^n (2n-1)!! / r^(2n+1) */
  double base = 1.0 / r;
  for (int n = 0; n <= order; ++n) {
    H[HI(n, 0, 0, 0)] = base;
    base *= -(double)(2 * n + 1) / r2;
  }
  for (int s = 1; s <= order; ++s) {
    for (int n = 0; n + s <= order; ++n) {
      for (int t = s; t >= 0; --t)
        for (int u = s - t; u >= 0; --u) {
          int v = s - t - u;
          double val;
          if (t > 0) {
            val = X * H[HI(n + 1, t - 1, u, v)];
            if (t > 1) val += (double)(t - 1) * H[HI(n + 1, t - 2, u, v)];
          } else if (u > 0) {
            val = Y * H[HI(n + 1, t, u - 1, v)];
            if (u > 1) val += (double)(u - 1) * H[HI(n + 1, t, u - 2, v)];
          } else {
            val = Z * H[HI(n + 1, t, u, v - 1)];
            if (v > 1) val += (double)(v - 1) * H[HI(n + 1, t, u, v - 2)];
          }
          H[HI(n, t, u, v)] = val;
        }
    }
  }
  for (int k = 0; k < oracle_ncoef(order); ++k) {
    const int* g = ix->mi[k];
    D[k] = -H[HI(0, g[0], g[1], g[2])]; /* g = -1/r */
  }
#undef HI
  free(H);
}

int oracle_dtensor(const double* R, int order, double* D) {
  if (order < 0 || order > OR_MAXP) return -1;
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, order);
  or_dtensor_ix(ix, R, order, D);
  free(ix);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Single translation operators (each on one expansion).                    */
/* ------------------------------------------------------------------------ */

/* M2M, Sec. 2.1 eq. M2M_general written per multi-index and moved from the
 * child centre to the parent centre:  with d = c_child - c_parent,
 *   M_alpha(parent) += sum_{beta <= alpha} C(alpha,beta) d^(alpha-beta) M_beta(child). */
static void or_m2m(const or_index* ix, const double* Mc, const double d[3], double* Mp) {
  for (int ka = 0; ka < ix->nc; ++ka) {
    const int* a = ix->mi[ka];
    double s = 0.0;
    for (int kb = 0; kb < ix->nc; ++kb) {
      const int* b = ix->mi[kb];
      if (b[0] > a[0] || b[1] > a[1] || b[2] > a[2]) continue;
      double w = 1.0;
#if ORACLE_MUTANT == 10 /* planted mistake: binomial coefficients dropped */
      for (int q = 0; q < 3; ++q) w *= or_ipow(d[q], a[q] - b[q]);
#else
      for (int q = 0; q < 3; ++q) w *= or_binom(a[q], b[q]) * or_ipow(d[q], a[q] - b[q]);
#endif
      s += w * Mc[kb];
    }
    Mp[ka] += s;
  }
}

/* M2L, Sec. 2.3 eq. M2L per multi-index, R = c_target - c_source (Q1). */
static void or_m2l(const or_index* ix, const double* M, const double R[3], double* L) {
  const int p = ix->p;
  double D[1000];
  or_dtensor_ix(ix, R, p, D);
  for (int kb = 0; kb < ix->nc; ++kb) {
    const int* b = ix->mi[kb];
    const int nb = b[0] + b[1] + b[2];
    double s = 0.0;
    for (int ka = 0; ka < ix->nc; ++ka) {
      const int* a = ix->mi[ka];
      const int na = a[0] + a[1] + a[2];
#if ORACLE_MUTANT == 8 /* planted mistake: the two order limits applied to the wrong sides */
      if (na + nb > p || na > ix->lo || nb > ix->mo) continue;
#else
      if (na + nb > p || na > ix->mo || nb > ix->lo) continue;
#endif
      const int kg = ix->lut[a[0] + b[0]][a[1] + b[1]][a[2] + b[2]];
      double afact = or_fact(a[0]) * or_fact(a[1]) * or_fact(a[2]);
      double sgn = (na & 1) ? -1.0 : 1.0;
#if ORACLE_MUTANT == 1 /* planted mistake: R taken as source - target */
      sgn *= ((na + nb) & 1) ? -1.0 : 1.0;
#endif
#if ORACLE_MUTANT == 2 /* planted mistake: the 1/alpha! factor dropped */
      afact = 1.0;
#endif
      s += sgn / afact * D[kg] * M[ka];
    }
    L[kb] += s;
  }
}

/* M2P, the paper's final-stage evaluation (Sec. 4): the potential of the
 * multipoles M about a source centre at a point R = x - c_source, i.e. eq. M2L
 * with beta = 0 evaluated at the point itself:
 *   phi(x) = sum_alpha (-1)^|alpha| / alpha! D_alpha(R) M_alpha. */
static double or_m2p(const or_index* ix, const double* M, const double R[3]) {
  double D[1000];
  or_dtensor_ix(ix, R, ix->p, D);
  double s = 0.0;
  for (int ka = 0; ka < ix->nc; ++ka) {
    const int* a = ix->mi[ka];
    const int na = a[0] + a[1] + a[2];
    if (na > ix->mo) continue;
    const double afact = or_fact(a[0]) * or_fact(a[1]) * or_fact(a[2]);
#if ORACLE_MUTANT == 7 /* planted mistake: M2P without the (-1)^|alpha| factor */
    s += 1.0 / afact * D[ka] * M[ka];
#else
    s += ((na & 1) ? -1.0 : 1.0) / afact * D[ka] * M[ka];
#endif
  }
  return s;
}

/* L2L, Sec. 2.3 eq. L2L, a = c_child - c_parent:
 *   L_beta(child) += sum_{gamma >= beta} a^(gamma-beta)/(gamma-beta)! L_gamma(parent). */
static void or_l2l(const or_index* ix, const double* Lp, const double a[3], double* Lc) {
  for (int kb = 0; kb < ix->nc; ++kb) {
    const int* b = ix->mi[kb];
    double s = 0.0;
    for (int kg = 0; kg < ix->nc; ++kg) {
      const int* g = ix->mi[kg];
      if (g[0] < b[0] || g[1] < b[1] || g[2] < b[2]) continue;
      double w = 1.0;
      for (int q = 0; q < 3; ++q) {
        double aq = a[q];
#if ORACLE_MUTANT == 3 /* planted mistake: displacement taken parent - child */
        aq = -aq;
#endif
        w *= or_ipow(aq, g[q] - b[q]) / or_fact(g[q] - b[q]);
      }
      s += w * Lp[kg];
    }
    Lc[kb] += s;
  }
}

/* L2P (Sec. 2.3, the final evaluation of the local expansion). */
static double or_l2p(const or_index* ix, const double* L, const double e[3]) {
  double s = 0.0;
  for (int k = 0; k < ix->nc; ++k) {
    const int* b = ix->mi[k];
    double w = 1.0;
#if ORACLE_MUTANT == 11 /* planted mistake: the 1/beta! factor dropped */
    for (int q = 0; q < 3; ++q) w *= or_ipow(e[q], b[q]);
#else
    for (int q = 0; q < 3; ++q) w *= or_ipow(e[q], b[q]) / or_fact(b[q]);
#endif
    s += w * L[k];
  }
  return s;
}

/* Gradient of the local expansion (the derivative of L2P): d/de_q of
 * sum_beta L_beta e^beta / beta! = sum_{beta_q >= 1} L_beta e^(beta - e_q) / (beta - e_q)!.
 * Used by the analytic acceleration (the force read off the expansions). */
static void or_l2p_grad(const or_index* ix, const double* L, const double e[3], double g[3]) {
  g[0] = g[1] = g[2] = 0.0;
  for (int k = 0; k < ix->nc; ++k) {
    const int* b = ix->mi[k];
    for (int q = 0; q < 3; ++q) {
      if (b[q] == 0) continue;
      double w = 1.0;
      for (int r = 0; r < 3; ++r) {
        const int pw = b[r] - (r == q);
#if ORACLE_MUTANT == 15 /* planted mistake: the undifferentiated factorials kept */
        w *= or_ipow(e[r], pw) / or_fact(b[r]);
#else
        w *= or_ipow(e[r], pw) / or_fact(pw);
#endif
      }
      g[q] += w * L[k];
    }
  }
}

/* Public single-operator entry points (used by the operator pins). */
int oracle_m2m(const double* Mc, const double* d, int p, double* Mp) {
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  or_m2m(ix, Mc, d, Mp);
  free(ix);
  return 0;
}
int oracle_m2l(const double* M, const double* R, int p, double* L) {
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  or_m2l(ix, M, R, L);
  free(ix);
  return 0;
}
int oracle_l2l(const double* Lp, const double* a, int p, double* Lc) {
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  or_l2l(ix, Lp, a, Lc);
  free(ix);
  return 0;
}
double oracle_l2p(const double* L, const double* e, int p) {
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  double v = or_l2p(ix, L, e);
  free(ix);
  return v;
}

/* Near-field Green's function, Sec. 2.3 eq. direct, in cell units. */
static double or_g(double rx, double ry, double rz) {
  double r = sqrt(rx * rx + ry * ry + rz * rz);
  if (r <= 1.0) return -1.0; /* |r| <= dx: -1/dx (only the self cell on a grid) */
  return -1.0 / r;
}

/* Gradient in x of g(x - y) for the cell pair force: r / |r|^3 with r = x - y
 * for distinct cells, and no self force (the softened kernel is constant at
 * the self cell; reading of the force between distinct cells). */
static void or_grad_g(double rx, double ry, double rz, double g[3]) {
  const double r2 = rx * rx + ry * ry + rz * rz;
  if (r2 == 0.0) {
    g[0] = g[1] = g[2] = 0.0;
    return;
  }
  const double inv = 1.0 / (r2 * sqrt(r2));
#if ORACLE_MUTANT == 6 /* planted mistake: near-field force pointing away from the mass */
  g[0] = -rx * inv, g[1] = -ry * inv, g[2] = -rz * inv;
#else
  g[0] = rx * inv, g[1] = ry * inv, g[2] = rz * inv;
#endif
}

/* ------------------------------------------------------------------------ */
/* Hierarchy (Sec. 2; Fig. 1).                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n[3];
  long nbox;
  double h; /* box side in cells */
} or_level;

typedef struct {
  int N[3], b, p, L; /* L = index of the leaf level */
  or_level lev[OR_MAXLEV];
} or_hier;

static int or_hier_init(or_hier* H, int nx, int ny, int nz, int b, int p) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || b <= 0) return -1;
  if (nx % b || ny % b || nz % b) return -1;
  if (p < 0 || p > OR_MAXP) return -1;
  H->N[0] = nx;
  H->N[1] = ny;
  H->N[2] = nz;
  H->b = b;
  H->p = p;
  int ext[OR_MAXLEV][3];
  int cnt = 0;
  ext[0][0] = nx / b;
  ext[0][1] = ny / b;
  ext[0][2] = nz / b;
  cnt = 1;
  while (ext[cnt - 1][0] > 1 || ext[cnt - 1][1] > 1 || ext[cnt - 1][2] > 1) {
    for (int q = 0; q < 3; ++q) ext[cnt][q] = (ext[cnt - 1][q] + 1) / 2;
    ++cnt;
    if (cnt >= OR_MAXLEV) return -1;
  }
  H->L = cnt - 1;
  for (int l = 0; l <= H->L; ++l) {
    int src = H->L - l; /* ext[0] is the leaf */
    for (int q = 0; q < 3; ++q) H->lev[l].n[q] = ext[src][q];
    H->lev[l].nbox = (long)ext[src][0] * ext[src][1] * ext[src][2];
    H->lev[l].h = (double)b * (double)(1L << (H->L - l));
  }
  return 0;
}

/* Level extents for tests: writes 3*(L+1) ints (level 0 first); returns L. */
int oracle_levels(int nx, int ny, int nz, int b, int* out) {
  or_hier H;
  if (or_hier_init(&H, nx, ny, nz, b, 0)) return -1;
  for (int l = 0; l <= H.L; ++l)
    for (int q = 0; q < 3; ++q) out[3 * l + q] = H.lev[l].n[q];
  return H.L;
}

static long or_bidx(const or_level* lv, int i, int j, int k) {
  return ((long)k * lv->n[1] + j) * lv->n[0] + i;
}

static void or_bcentre(const or_level* lv, int i, int j, int k, double c[3]) {
  c[0] = (i + 0.5) * lv->h;
  c[1] = (j + 0.5) * lv->h;
  c[2] = (k + 0.5) * lv->h;
}

/* Interaction list of target box (i,j,k) at level l >= 1 (Sec. 2.2):
 * children of the parent's 27 neighbours (clipped) that are at Chebyshev
 * distance >= 2 from the target.  Writes box triples; returns the count. */
static int or_ilist(const or_hier* H, int l, int i, int j, int k, int (*out)[3]) {
  const or_level* pl = &H->lev[l - 1];
  const or_level* cl = &H->lev[l];
  int cnt = 0;
  int pi = i / 2, pj = j / 2, pk = k / 2;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int qi = pi + dx, qj = pj + dy, qk = pk + dz;
        if (qi < 0 || qj < 0 || qk < 0 || qi >= pl->n[0] || qj >= pl->n[1] || qk >= pl->n[2]) continue;
        for (int cz = 0; cz < 2; ++cz)
          for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
              int si = 2 * qi + cx, sj = 2 * qj + cy, sk = 2 * qk + cz;
              if (si >= cl->n[0] || sj >= cl->n[1] || sk >= cl->n[2]) continue;
              int di = abs(si - i), dj = abs(sj - j), dk = abs(sk - k);
              int cheb = di > dj ? di : dj;
              cheb = cheb > dk ? cheb : dk;
#if ORACLE_MUTANT == 4 /* planted mistake: near neighbours also taken into the list */
              if (cheb < 1) continue;
#else
              if (cheb < 2) continue;
#endif
              out[cnt][0] = si;
              out[cnt][1] = sj;
              out[cnt][2] = sk;
              ++cnt;
            }
      }
  return cnt;
}

/* Interaction-list size of one target, for the Sec. 2.2 geometry pin. */
int oracle_ilist_count(int nx, int ny, int nz, int b, int level, int i, int j, int k) {
  or_hier H;
  if (or_hier_init(&H, nx, ny, nz, b, 0)) return -1;
  if (level < 1 || level > H.L) return -1;
  int buf[216][3];
  return or_ilist(&H, level, i, j, k, buf);
}

/* ------------------------------------------------------------------------ */
/* Upward pass.                                                             */
/* ------------------------------------------------------------------------ */

/* P2M about an arbitrary centre for the cell block [lo, lo+ext) (Sec. 2.1
 * eq. multipole, moments about c).  Cells outside the grid contribute 0. */
static void or_p2m_region(const or_index* ix, const double* rho, const int N[3], const int lo[3],
                          const int ext[3], const double c[3], double* M) {
  for (int k = 0; k < ix->nc; ++k) M[k] = 0.0;
  for (int z = lo[2]; z < lo[2] + ext[2]; ++z) {
    if (z < 0 || z >= N[2]) continue;
    for (int y = lo[1]; y < lo[1] + ext[1]; ++y) {
      if (y < 0 || y >= N[1]) continue;
      for (int x = lo[0]; x < lo[0] + ext[0]; ++x) {
        if (x < 0 || x >= N[0]) continue;
        double m = rho[((long)z * N[1] + y) * N[0] + x];
        if (m == 0.0) continue;
#if ORACLE_MUTANT == 9 /* planted mistake: cells placed at their lower corners */
        double e[3] = {x - c[0], y - c[1], z - c[2]};
#else
        double e[3] = {x + 0.5 - c[0], y + 0.5 - c[1], z + 0.5 - c[2]};
#endif
        for (int k = 0; k < ix->nc; ++k) {
          const int* a = ix->mi[k];
          M[k] += m * or_ipow(e[0], a[0]) * or_ipow(e[1], a[1]) * or_ipow(e[2], a[2]);
        }
      }
    }
  }
}

int oracle_p2m_region(const double* rho, int nx, int ny, int nz, const int* lo, const int* ext,
                      const double* c, int p, double* M) {
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  int N[3] = {nx, ny, nz};
  or_p2m_region(ix, rho, N, lo, ext, c, M);
  free(ix);
  return 0;
}

/* Full centred upward pass: M[l] for every level (Sec. 2.1). */
static double** or_upward(const or_hier* H, const or_index* ix, const double* rho) {
  const int nc = ix->nc;
  double** M = (double**)calloc(H->L + 1, sizeof(double*));
  for (int l = 0; l <= H->L; ++l) M[l] = (double*)calloc((size_t)H->lev[l].nbox * nc, sizeof(double));
  /* P2M per leaf box */
  const or_level* lf = &H->lev[H->L];
#pragma omp parallel for schedule(dynamic, 16)
  for (long bi = 0; bi < lf->nbox; ++bi) {
    int i = (int)(bi % lf->n[0]);
    int j = (int)((bi / lf->n[0]) % lf->n[1]);
    int k = (int)(bi / ((long)lf->n[0] * lf->n[1]));
    int lo[3] = {i * H->b, j * H->b, k * H->b};
    int ext[3] = {H->b, H->b, H->b};
    double c[3];
    or_bcentre(lf, i, j, k, c);
    or_p2m_region(ix, rho, H->N, lo, ext, c, M[H->L] + bi * nc);
  }
  /* M2M child -> parent */
  for (int l = H->L - 1; l >= 0; --l) {
    const or_level* pl = &H->lev[l];
    const or_level* cl = &H->lev[l + 1];
#pragma omp parallel for schedule(dynamic, 16)
    for (long bi = 0; bi < pl->nbox; ++bi) {
      int i = (int)(bi % pl->n[0]);
      int j = (int)((bi / pl->n[0]) % pl->n[1]);
      int k = (int)(bi / ((long)pl->n[0] * pl->n[1]));
      double cp[3];
      or_bcentre(pl, i, j, k, cp);
      for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
          for (int cx = 0; cx < 2; ++cx) {
            int si = 2 * i + cx, sj = 2 * j + cy, sk = 2 * k + cz;
            if (si >= cl->n[0] || sj >= cl->n[1] || sk >= cl->n[2]) continue;
            double cc[3];
            or_bcentre(cl, si, sj, sk, cc);
            double d[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};
            or_m2m(ix, M[l + 1] + or_bidx(cl, si, sj, sk) * nc, d, M[l] + bi * nc);
          }
    }
  }
  return M;
}

/* The paper's own upward route (Sec. 2.1): moments about the origin summed
 * term by term up the hierarchy, then shifted to each cell centre with
 * eq. M2M_general (M'_alpha = sum_k C(alpha,k) (-a)^(alpha-k) M_k).
 * Returns the level-`level` moments in Mout (nbox * nc). */
int oracle_upward_origin(const double* rho, int nx, int ny, int nz, int b, int p, int level, double* Mout) {
  or_hier H;
  if (or_hier_init(&H, nx, ny, nz, b, p)) return -1;
  if (level < 0 || level > H.L) return -1;
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  const int nc = ix->nc;
  const or_level* lv = &H.lev[level];
  /* accumulate origin moments straight from the cells covered by each box */
  double* M0 = (double*)calloc((size_t)lv->nbox * nc, sizeof(double));
  double origin[3] = {0.0, 0.0, 0.0};
  int boxc = (int)lv->h;
  for (long bi = 0; bi < lv->nbox; ++bi) {
    int i = (int)(bi % lv->n[0]);
    int j = (int)((bi / lv->n[0]) % lv->n[1]);
    int k = (int)(bi / ((long)lv->n[0] * lv->n[1]));
    /* term-by-term sum of the leaf cells' origin moments */
    int lo[3] = {i * boxc, j * boxc, k * boxc};
    int ext[3] = {boxc, boxc, boxc};
    or_p2m_region(ix, rho, H.N, lo, ext, origin, M0 + bi * nc);
    /* shift origin -> centre a: eq. M2M_general */
    double a[3];
    or_bcentre(lv, i, j, k, a);
    double na[3] = {-a[0], -a[1], -a[2]};
    double* out = Mout + bi * nc;
    for (int q = 0; q < nc; ++q) out[q] = 0.0;
    or_m2m(ix, M0 + bi * nc, na, out);
  }
  free(M0);
  free(ix);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Downward pass and leaf evaluation (Sec. 2.3).                            */
/* ------------------------------------------------------------------------ */

/* Downward pass; with leaf_m2l = 0 the leaf level gets only its parent's
 * local expansion (the final-stage M2P evaluates the leaf interaction list). */
static double** or_downward_ex(const or_hier* H, const or_index* ix, double** M, int leaf_m2l) {
  const int nc = ix->nc;
  double** L = (double**)calloc(H->L + 1, sizeof(double*));
  for (int l = 0; l <= H->L; ++l) L[l] = (double*)calloc((size_t)H->lev[l].nbox * nc, sizeof(double));
  for (int l = 1; l <= H->L; ++l) {
    const or_level* cl = &H->lev[l];
    const or_level* pl = &H->lev[l - 1];
#pragma omp parallel for schedule(dynamic, 4)
    for (long bi = 0; bi < cl->nbox; ++bi) {
      int i = (int)(bi % cl->n[0]);
      int j = (int)((bi / cl->n[0]) % cl->n[1]);
      int k = (int)(bi / ((long)cl->n[0] * cl->n[1]));
      double ct[3], cp[3];
      or_bcentre(cl, i, j, k, ct);
      or_bcentre(pl, i / 2, j / 2, k / 2, cp);
      double* Lt = L[l] + bi * nc;
      /* far field: parent's local expansion moved to this centre (eq. L2L) */
      double a[3] = {ct[0] - cp[0], ct[1] - cp[1], ct[2] - cp[2]};
      or_l2l(ix, L[l - 1] + or_bidx(pl, i / 2, j / 2, k / 2) * nc, a, Lt);
      /* intermediate field: M2L over the interaction list (eq. M2L) */
      if (l == H->L && !leaf_m2l) continue;
      int il[216][3];
      int n = or_ilist(H, l, i, j, k, il);
      for (int s = 0; s < n; ++s) {
        double cs[3];
        or_bcentre(cl, il[s][0], il[s][1], il[s][2], cs);
        double R[3] = {ct[0] - cs[0], ct[1] - cs[1], ct[2] - cs[2]};
        or_m2l(ix, M[l] + or_bidx(cl, il[s][0], il[s][1], il[s][2]) * nc, R, Lt);
      }
    }
  }
  return L;
}

static double** or_downward(const or_hier* H, const or_index* ix, double** M) {
  return or_downward_ex(H, ix, M, 1);
}

/* Near field of one cell: all cells of the leaf boxes at Chebyshev distance
 * <= 1 from its box (Fig. 1, right panel; eq. direct). */
static double or_near_cell(const or_hier* H, const double* rho, int x, int y, int z) {
  const or_level* lf = &H->lev[H->L];
  const int b = H->b;
  int bi = x / b, bj = y / b, bk = z / b;
  double s = 0.0;
  for (int qk = bk - 1; qk <= bk + 1; ++qk) {
    if (qk < 0 || qk >= lf->n[2]) continue;
    for (int qj = bj - 1; qj <= bj + 1; ++qj) {
      if (qj < 0 || qj >= lf->n[1]) continue;
      for (int qi = bi - 1; qi <= bi + 1; ++qi) {
        if (qi < 0 || qi >= lf->n[0]) continue;
#if ORACLE_MUTANT == 16 /* planted mistake: only the 6 face neighbours (edge and corner boxes dropped) */
        if (abs(qi - bi) + abs(qj - bj) + abs(qk - bk) > 1) continue;
#endif
        for (int sz = qk * b; sz < qk * b + b; ++sz)
          for (int sy = qj * b; sy < qj * b + b; ++sy)
            for (int sx = qi * b; sx < qi * b + b; ++sx) {
#if ORACLE_MUTANT == 5 /* planted mistake: self cell left out */
              if (sx == x && sy == y && sz == z) continue;
#endif
              double m = rho[((long)sz * H->N[1] + sy) * H->N[0] + sx];
              s += m * or_g((double)(x - sx), (double)(y - sy), (double)(z - sz));
            }
      }
    }
  }
  return s;
}

/* Gradient of the near-field potential of one cell (same near region). */
static void or_near_grad(const or_hier* H, const double* rho, int x, int y, int z, double out[3]) {
  const or_level* lf = &H->lev[H->L];
  const int b = H->b;
  int bi = x / b, bj = y / b, bk = z / b;
  out[0] = out[1] = out[2] = 0.0;
  for (int qk = bk - 1; qk <= bk + 1; ++qk) {
    if (qk < 0 || qk >= lf->n[2]) continue;
    for (int qj = bj - 1; qj <= bj + 1; ++qj) {
      if (qj < 0 || qj >= lf->n[1]) continue;
      for (int qi = bi - 1; qi <= bi + 1; ++qi) {
        if (qi < 0 || qi >= lf->n[0]) continue;
        for (int sz = qk * b; sz < qk * b + b; ++sz)
          for (int sy = qj * b; sy < qj * b + b; ++sy)
            for (int sx = qi * b; sx < qi * b + b; ++sx) {
              double m = rho[((long)sz * H->N[1] + sy) * H->N[0] + sx];
              double g[3];
              or_grad_g((double)(x - sx), (double)(y - sy), (double)(z - sz), g);
              for (int q = 0; q < 3; ++q) out[q] += m * g[q];
            }
      }
    }
  }
}

static void or_far_grad(const or_hier* H, const or_index* ix, double** L, int x, int y, int z, double g[3]) {
  const or_level* lf = &H->lev[H->L];
  int bi = x / H->b, bj = y / H->b, bk = z / H->b;
  double c[3];
  or_bcentre(lf, bi, bj, bk, c);
  double e[3] = {x + 0.5 - c[0], y + 0.5 - c[1], z + 0.5 - c[2]};
  or_l2p_grad(ix, L[H->L] + or_bidx(lf, bi, bj, bk) * ix->nc, e, g);
}

static double or_far_cell(const or_hier* H, const or_index* ix, double** L, int x, int y, int z) {
  const or_level* lf = &H->lev[H->L];
  int bi = x / H->b, bj = y / H->b, bk = z / H->b;
  double c[3];
  or_bcentre(lf, bi, bj, bk, c);
  double e[3] = {x + 0.5 - c[0], y + 0.5 - c[1], z + 0.5 - c[2]};
  return or_l2p(ix, L[H->L] + or_bidx(lf, bi, bj, bk) * ix->nc, e);
}

static void or_free_levels(const or_hier* H, double** A) {
  if (!A) return;
  for (int l = 0; l <= H->L; ++l) free(A[l]);
  free(A);
}

/* ------------------------------------------------------------------------ */
/* Force: 5-point finite-difference gradient (App. C), a = -grad(phi).       */
/* Interior 4th-order central; one cell from an edge 2nd-order central; at  */
/* the edge 2nd-order one-sided (reading Q9).                               */
/* ------------------------------------------------------------------------ */

static double or_fd_deriv(const double* f, long stride, int i, int n) {
  /* derivative along one axis in cell units at index i; f points at index 0 */
#define F(q) f[(long)(q) * stride]
  if (n == 1) return 0.0;
  if (n == 2) return F(1) - F(0);
#if ORACLE_MUTANT == 12 /* planted mistake: outer weights of the 5-point stencil with the wrong sign */
  if (i >= 2 && i <= n - 3) return (F(i + 2) + 8.0 * F(i + 1) - 8.0 * F(i - 1) - F(i - 2)) / 12.0;
#else
  if (i >= 2 && i <= n - 3) return (-F(i + 2) + 8.0 * F(i + 1) - 8.0 * F(i - 1) + F(i - 2)) / 12.0;
#endif
  if (i >= 1 && i <= n - 2) return (F(i + 1) - F(i - 1)) / 2.0;
  if (i == 0) return (-3.0 * F(0) + 4.0 * F(1) - F(2)) / 2.0;
  return (3.0 * F(n - 1) - 4.0 * F(n - 2) + F(n - 3)) / 2.0;
#undef F
}

/* accel[3][n]: a_q = -(1/dx) d phi / d x_q  (phi already physical) */
int oracle_fd_accel(const double* phi, int nx, int ny, int nz, double dx, double* accel) {
  const long n = (long)nx * ny * nz;
#pragma omp parallel for
  for (long c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    const double* rowx = phi + ((long)z * ny + y) * nx;
    const double* coly = phi + (long)z * ny * nx + x;
    const double* colz = phi + (long)y * nx + x;
    accel[c] = -or_fd_deriv(rowx, 1, x, nx) / dx;
    accel[n + c] = -or_fd_deriv(coly, nx, y, ny) / dx;
    accel[2 * n + c] = -or_fd_deriv(colz, (long)nx * ny, z, nz) / dx;
  }
  return 0;
}

/* Transpose of oracle_fd_accel: grad_phi += FD^T grad_accel (explicit
 * scatter of every stencil weight, not a reuse of the forward routine). */
static void or_fd_scatter(double* out, long stride, int i, int n, double w) {
#define O(q) out[(long)(q) * stride]
  if (n == 1) return;
  if (n == 2) {
    O(1) += w;
    O(0) -= w;
    return;
  }
  if (i >= 2 && i <= n - 3) {
    O(i + 2) += -w / 12.0;
    O(i + 1) += 8.0 * w / 12.0;
    O(i - 1) += -8.0 * w / 12.0;
    O(i - 2) += w / 12.0;
  } else if (i >= 1 && i <= n - 2) {
    O(i + 1) += w / 2.0;
    O(i - 1) -= w / 2.0;
  } else if (i == 0) {
    O(0) += -3.0 * w / 2.0;
    O(1) += 4.0 * w / 2.0;
#if ORACLE_MUTANT == 13 /* planted mistake: one-sided edge weight scattered with the wrong sign */
    O(2) += w / 2.0;
#else
    O(2) += -w / 2.0;
#endif
  } else {
    O(n - 1) += 3.0 * w / 2.0;
    O(n - 2) += -4.0 * w / 2.0;
    O(n - 3) += w / 2.0;
  }
#undef O
}

int oracle_fd_accel_adjoint(const double* gaccel, int nx, int ny, int nz, double dx, double* gphi) {
  const long n = (long)nx * ny * nz;
  for (long c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    or_fd_scatter(gphi + ((long)z * ny + y) * nx, 1, x, nx, -gaccel[c] / dx);
    or_fd_scatter(gphi + (long)z * ny * nx + x, nx, y, ny, -gaccel[n + c] / dx);
    or_fd_scatter(gphi + (long)y * nx + x, (long)nx * ny, z, nz, -gaccel[2 * n + c] / dx);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Whole solve.                                                             */
/* ------------------------------------------------------------------------ */

static void or_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * oracle_fmm: phi (and optionally accel[3][n], phi_far, phi_near) for a
 * density rho on an isolated nx*ny*nz grid; leaf boxes b^3, order p.
 * Optional exports: Mlev/Llev = moments / locals (cell units, about box
 * centres, canonical order) of level `exp_level` (nbox * ncoef doubles).
 * Returns 0 on success, -1 on bad arguments.
 */
int oracle_fmm(const double* rho, int nx, int ny, int nz, int b, int p, double dx, double G,
               double* phi, double* accel, double* phi_far, double* phi_near, int exp_level,
               double* Mlev, double* Llev, int nthreads) {
  or_hier H;
  if (or_hier_init(&H, nx, ny, nz, b, p)) return -1;
  or_set_threads(nthreads);
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  double** M = or_upward(&H, ix, rho);
  double** L = or_downward(&H, ix, M);
  const long n = (long)nx * ny * nz;
  const double scale = G * dx * dx;
#pragma omp parallel for schedule(dynamic, 64)
  for (long c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    double ff = or_far_cell(&H, ix, L, x, y, z);
    double nf = or_near_cell(&H, rho, x, y, z);
    phi[c] = scale * (ff + nf);
    if (phi_far) phi_far[c] = scale * ff;
    if (phi_near) phi_near[c] = scale * nf;
  }
  if (accel) oracle_fd_accel(phi, nx, ny, nz, dx, accel);
  if (exp_level >= 0 && exp_level <= H.L) {
    size_t cnt = (size_t)H.lev[exp_level].nbox * ix->nc;
    if (Mlev) memcpy(Mlev, M[exp_level], cnt * sizeof(double));
    if (Llev) memcpy(Llev, L[exp_level], cnt * sizeof(double));
  }
  or_free_levels(&H, M);
  or_free_levels(&H, L);
  free(ix);
  return 0;
}

/* O(N^2) direct sum with the same softened Green's function (eq. direct over
 * every cell pair): the brute-force reference the paper's App. B uses. */
int oracle_direct(const double* rho, int nx, int ny, int nz, double dx, double G, double* phi, int nthreads) {
  or_set_threads(nthreads);
  const long n = (long)nx * ny * nz;
  const double scale = G * dx * dx;
#pragma omp parallel for schedule(dynamic, 16)
  for (long c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    double s = 0.0;
    for (long d = 0; d < n; ++d) {
      double m = rho[d];
      if (m == 0.0) continue;
      int sx = (int)(d % nx), sy = (int)((d / nx) % ny), sz = (int)(d / ((long)nx * ny));
      s += m * or_g((double)(x - sx), (double)(y - sy), (double)(z - sz));
    }
    phi[c] = scale * s;
  }
  return 0;
}

/* Potential (and optionally accel) at a sample of cells, at any grid size:
 * the full upward pass, then for each sampled cell the chain of local
 * expansions of its ancestors (eq. L2L + eq. M2L), L2P and the near field.
 * accel needs phi at the +-2 stencil neighbours, evaluated the same way. */
static void or_local_chain(const or_hier* H, const or_index* ix, double** M, int l, int i, int j, int k, double* Lout) {
  const int nc = ix->nc;
  for (int q = 0; q < nc; ++q) Lout[q] = 0.0;
  if (l == 0) return;
  double* Lp = (double*)calloc(nc, sizeof(double));
  or_local_chain(H, ix, M, l - 1, i / 2, j / 2, k / 2, Lp);
  const or_level* cl = &H->lev[l];
  const or_level* pl = &H->lev[l - 1];
  double ct[3], cp[3];
  or_bcentre(cl, i, j, k, ct);
  or_bcentre(pl, i / 2, j / 2, k / 2, cp);
  double a[3] = {ct[0] - cp[0], ct[1] - cp[1], ct[2] - cp[2]};
  or_l2l(ix, Lp, a, Lout);
  free(Lp);
  int il[216][3];
  int n = or_ilist(H, l, i, j, k, il);
  for (int s = 0; s < n; ++s) {
    double cs[3];
    or_bcentre(cl, il[s][0], il[s][1], il[s][2], cs);
    double R[3] = {ct[0] - cs[0], ct[1] - cs[1], ct[2] - cs[2]};
    or_m2l(ix, M[l] + or_bidx(cl, il[s][0], il[s][1], il[s][2]) * nc, R, Lout);
  }
}

static double or_phi_cell_sampled(const or_hier* H, const or_index* ix, double** M, const double* rho, int x, int y,
                                  int z) {
  const or_level* lf = &H->lev[H->L];
  int bi = x / H->b, bj = y / H->b, bk = z / H->b;
  double* Lb = (double*)malloc(sizeof(double) * ix->nc);
  or_local_chain(H, ix, M, H->L, bi, bj, bk, Lb);
  double c[3];
  or_bcentre(lf, bi, bj, bk, c);
  double e[3] = {x + 0.5 - c[0], y + 0.5 - c[1], z + 0.5 - c[2]};
  double ff = or_l2p(ix, Lb, e);
  free(Lb);
  return ff + or_near_cell(H, rho, x, y, z);
}

int oracle_fmm_sample(const double* rho, int nx, int ny, int nz, int b, int p, double dx, double G, long nsample,
                      const long* cells, double* phi_out, double* accel_out /* [nsample][3] or NULL */,
                      int nthreads) {
  or_hier H;
  if (or_hier_init(&H, nx, ny, nz, b, p)) return -1;
  or_set_threads(nthreads);
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  double** M = or_upward(&H, ix, rho);
  const double scale = G * dx * dx;
  const int N[3] = {nx, ny, nz};
#pragma omp parallel for schedule(dynamic, 1)
  for (long s = 0; s < nsample; ++s) {
    long c = cells[s];
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    phi_out[s] = scale * or_phi_cell_sampled(&H, ix, M, rho, x, y, z);
    if (accel_out) {
      int pos[3] = {x, y, z};
      for (int q = 0; q < 3; ++q) {
        /* phi along axis q at the +-2 window the FD rule reads */
        int n = N[q], i = pos[q];
        double* line = (double*)calloc((size_t)n, sizeof(double));
        for (int v = i - 2; v <= i + 2; ++v) {
          if (v < 0 || v >= n) continue;
          int pp[3] = {x, y, z};
          pp[q] = v;
          line[v] = scale * or_phi_cell_sampled(&H, ix, M, rho, pp[0], pp[1], pp[2]);
        }
        accel_out[3 * s + q] = -or_fd_deriv(line, 1, i, n) / dx;
        free(line);
      }
    }
  }
  or_free_levels(&H, M);
  free(ix);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint: the explicit transpose of every step of oracle_fmm, composed in  */
/* reverse order (not the forward applied again), so that the symmetry of  */
/* the FMM operator is something the tests check, not something assumed.   */
/*   forward:  phi = s * (Near + L2P L2L^k M2L M2M^k P2M) rho, s = G dx^2    */
/*             accel = -(1/dx) FD phi                                       */
/*   adjoint:  grad_rho = s * (Near^T + P2M^T M2M^T.. M2L^T .. L2L^T L2P^T) w */
/*             w = grad_phi + FD^T(-(1/dx) grad_accel)                       */
/* ------------------------------------------------------------------------ */

/* analytic = 0: the force is the 5-point stencil of phi, so grad_accel joins
 * the source w through FD^T.  analytic = 1: the force is the analytic one of
 * oracle_fmm_accel, accel = -G dx (grad far + grad near); with v = -grad_accel
 * / dx (the factor relative to the potential's G dx^2) its transpose adds
 * grad-L2P^T v to the leaf Lam (sum_q v_q e^(beta - e_q) / (beta - e_q)!)
 * and, per source cell c, sum over the targets t whose near region holds c of
 * v(t) . grad g(x_t - x_c). */
static int or_adjoint(const double* gphi, const double* gaccel, int analytic, int nx, int ny, int nz, int b, int p,
                      double dx, double G, double* grho, int nthreads) {
  or_hier H;
  if (or_hier_init(&H, nx, ny, nz, b, p)) return -1;
  or_set_threads(nthreads);
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  const int nc = ix->nc;
  const long n = (long)nx * ny * nz;
  const double scale = G * dx * dx;
  double* w = (double*)malloc(sizeof(double) * n);
  memcpy(w, gphi, sizeof(double) * n);
  double* v = NULL; /* analytic: v[3][n] = -grad_accel / dx */
  if (gaccel && !analytic) oracle_fd_accel_adjoint(gaccel, nx, ny, nz, dx, w);
  if (gaccel && analytic) {
    v = (double*)malloc(sizeof(double) * 3 * n);
    for (long c = 0; c < 3 * n; ++c) v[c] = -gaccel[c] / dx;
  }
  /* L2P^T: Lam_beta(B) = sum_{i in B} w_i e_i^beta / beta! */
  double** Lam = (double**)calloc(H.L + 1, sizeof(double*));
  double** Mu = (double**)calloc(H.L + 1, sizeof(double*));
  for (int l = 0; l <= H.L; ++l) {
    Lam[l] = (double*)calloc((size_t)H.lev[l].nbox * nc, sizeof(double));
    Mu[l] = (double*)calloc((size_t)H.lev[l].nbox * nc, sizeof(double));
  }
  const or_level* lf = &H.lev[H.L];
  for (long c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    int bi = x / b, bj = y / b, bk = z / b;
    double cc[3];
    or_bcentre(lf, bi, bj, bk, cc);
    double e[3] = {x + 0.5 - cc[0], y + 0.5 - cc[1], z + 0.5 - cc[2]};
    double* La = Lam[H.L] + or_bidx(lf, bi, bj, bk) * nc;
    for (int k = 0; k < nc; ++k) {
      const int* be = ix->mi[k];
      double t = 1.0;
#if ORACLE_MUTANT == 14 /* planted mistake: L2P^T without the 1/beta! factor */
      for (int q = 0; q < 3; ++q) t *= or_ipow(e[q], be[q]);
#else
      for (int q = 0; q < 3; ++q) t *= or_ipow(e[q], be[q]) / or_fact(be[q]);
#endif
      La[k] += w[c] * t;
    }
    if (v) {
      for (int k = 0; k < nc; ++k) {
        /* grad-L2P^T: d/de_q (e^beta / beta!) = e^(beta - e_q) / (beta - e_q)! */
        const int* be = ix->mi[k];
        double s = 0.0;
        for (int q = 0; q < 3; ++q) {
          if (be[q] == 0) continue;
          double t = 1.0;
          for (int r = 0; r < 3; ++r) {
            const int pw = be[r] - (r == q);
            t *= or_ipow(e[r], pw) / or_fact(pw);
          }
          s += v[q * n + c] * t;
        }
        La[k] += s;
      }
    }
  }
  /* walk levels fine -> coarse: at level l, M2L^T scatters Lam(T) into
   * Mu(S) for S in IL(T); L2L^T moves Lam(T) into Lam(parent). */
  for (int l = H.L; l >= 1; --l) {
    const or_level* cl = &H.lev[l];
    const or_level* pl = &H.lev[l - 1];
    for (long bi = 0; bi < cl->nbox; ++bi) {
      int i = (int)(bi % cl->n[0]);
      int j = (int)((bi / cl->n[0]) % cl->n[1]);
      int k = (int)(bi / ((long)cl->n[0] * cl->n[1]));
      double ct[3], cp[3];
      or_bcentre(cl, i, j, k, ct);
      or_bcentre(pl, i / 2, j / 2, k / 2, cp);
      const double* La = Lam[l] + bi * nc;
      /* M2L^T: Mu_alpha(S) += sum_beta (-1)^|alpha|/alpha! D_{alpha+beta}(R) Lam_beta(T) */
      int il[216][3];
      int cnt = or_ilist(&H, l, i, j, k, il);
      double D[1000];
      for (int s = 0; s < cnt; ++s) {
        double cs[3];
        or_bcentre(cl, il[s][0], il[s][1], il[s][2], cs);
        double R[3] = {ct[0] - cs[0], ct[1] - cs[1], ct[2] - cs[2]};
        or_dtensor_ix(ix, R, p, D);
        double* Ms = Mu[l] + or_bidx(cl, il[s][0], il[s][1], il[s][2]) * nc;
        for (int ka = 0; ka < nc; ++ka) {
          const int* a = ix->mi[ka];
          int na = a[0] + a[1] + a[2];
          double afact = or_fact(a[0]) * or_fact(a[1]) * or_fact(a[2]);
          double sgn = (na & 1) ? -1.0 : 1.0;
          double acc = 0.0;
          for (int kb = 0; kb < nc; ++kb) {
            const int* be = ix->mi[kb];
            if (na + be[0] + be[1] + be[2] > p) continue;
            acc += D[ix->lut[a[0] + be[0]][a[1] + be[1]][a[2] + be[2]]] * La[kb];
          }
          Ms[ka] += sgn / afact * acc;
        }
      }
      /* L2L^T: Lam_gamma(P) += sum_{beta <= gamma} a^(gamma-beta)/(gamma-beta)! Lam_beta(T) */
      double a[3] = {ct[0] - cp[0], ct[1] - cp[1], ct[2] - cp[2]};
      double* Lp = Lam[l - 1] + or_bidx(pl, i / 2, j / 2, k / 2) * nc;
      for (int kg = 0; kg < nc; ++kg) {
        const int* g = ix->mi[kg];
        double acc = 0.0;
        for (int kb = 0; kb < nc; ++kb) {
          const int* be = ix->mi[kb];
          if (be[0] > g[0] || be[1] > g[1] || be[2] > g[2]) continue;
          double t = 1.0;
          for (int q = 0; q < 3; ++q) t *= or_ipow(a[q], g[q] - be[q]) / or_fact(g[q] - be[q]);
          acc += t * La[kb];
        }
        Lp[kg] += acc;
      }
    }
  }
  /* M2M^T coarse -> fine: Mu_beta(C) += sum_{alpha >= beta} C(alpha,beta) d^(alpha-beta) Mu_alpha(P) */
  for (int l = 0; l < H.L; ++l) {
    const or_level* pl = &H.lev[l];
    const or_level* cl = &H.lev[l + 1];
    for (long bi = 0; bi < cl->nbox; ++bi) {
      int i = (int)(bi % cl->n[0]);
      int j = (int)((bi / cl->n[0]) % cl->n[1]);
      int k = (int)(bi / ((long)cl->n[0] * cl->n[1]));
      double cc[3], cp[3];
      or_bcentre(cl, i, j, k, cc);
      or_bcentre(pl, i / 2, j / 2, k / 2, cp);
      double d[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};
      const double* Mp = Mu[l] + or_bidx(pl, i / 2, j / 2, k / 2) * nc;
      double* Mc = Mu[l + 1] + bi * nc;
      for (int kb = 0; kb < nc; ++kb) {
        const int* be = ix->mi[kb];
        double acc = 0.0;
        for (int ka = 0; ka < nc; ++ka) {
          const int* a = ix->mi[ka];
          if (be[0] > a[0] || be[1] > a[1] || be[2] > a[2]) continue;
          double t = 1.0;
          for (int q = 0; q < 3; ++q) t *= or_binom(a[q], be[q]) * or_ipow(d[q], a[q] - be[q]);
          acc += t * Mp[ka];
        }
        Mc[kb] += acc;
      }
    }
  }
  /* P2M^T + Near^T per source cell */
#pragma omp parallel for schedule(dynamic, 64)
  for (long c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    int bi = x / b, bj = y / b, bk = z / b;
    double cc[3];
    or_bcentre(lf, bi, bj, bk, cc);
    double e[3] = {x + 0.5 - cc[0], y + 0.5 - cc[1], z + 0.5 - cc[2]};
    const double* Ms = Mu[H.L] + or_bidx(lf, bi, bj, bk) * nc;
    double far = 0.0;
    for (int k = 0; k < nc; ++k) {
      const int* a = ix->mi[k];
      far += Ms[k] * or_ipow(e[0], a[0]) * or_ipow(e[1], a[1]) * or_ipow(e[2], a[2]);
    }
    /* Near^T: targets t whose near region holds this cell, weight g(x_t - x_c) */
    double nearv = 0.0;
    for (int qk = bk - 1; qk <= bk + 1; ++qk) {
      if (qk < 0 || qk >= lf->n[2]) continue;
      for (int qj = bj - 1; qj <= bj + 1; ++qj) {
        if (qj < 0 || qj >= lf->n[1]) continue;
        for (int qi = bi - 1; qi <= bi + 1; ++qi) {
          if (qi < 0 || qi >= lf->n[0]) continue;
          for (int tz = qk * b; tz < qk * b + b; ++tz)
            for (int ty = qj * b; ty < qj * b + b; ++ty)
              for (int tx = qi * b; tx < qi * b + b; ++tx) {
                const long t = ((long)tz * ny + ty) * nx + tx;
                nearv += w[t] * or_g((double)(tx - x), (double)(ty - y), (double)(tz - z));
                if (v) {
                  double gg[3];
#if ORACLE_MUTANT == 17 /* planted mistake: transposed pair force taken from source to target */
                  or_grad_g((double)(x - tx), (double)(y - ty), (double)(z - tz), gg);
#else
                  or_grad_g((double)(tx - x), (double)(ty - y), (double)(tz - z), gg);
#endif
                  nearv += v[t] * gg[0] + v[n + t] * gg[1] + v[2 * n + t] * gg[2];
                }
              }
        }
      }
    }
    grho[c] = scale * (far + nearv);
  }
  or_free_levels(&H, Lam);
  or_free_levels(&H, Mu);
  free(w);
  free(v);
  free(ix);
  return 0;
}

int oracle_adjoint(const double* gphi, const double* gaccel, int nx, int ny, int nz, int b, int p, double dx,
                   double G, double* grho, int nthreads) {
  return or_adjoint(gphi, gaccel, 0, nx, ny, nz, b, p, dx, G, grho, nthreads);
}

/* Transpose of (phi, analytic accel): grad_rho from grad_phi and the
 * gradient with respect to oracle_fmm_accel's force. */
int oracle_adjoint_analytic(const double* gphi, const double* gaccel, int nx, int ny, int nz, int b, int p, double dx,
                            double G, double* grho, int nthreads) {
  return or_adjoint(gphi, gaccel, 1, nx, ny, nz, b, p, dx, G, grho, nthreads);
}

/* Gradient of the M2P evaluation of Sec. 4's final stage with respect to the
 * target point.  d/dx_q D_alpha(x - c) = D_{alpha + e_q}(x - c), so
 *   d phi / dx_q = sum_alpha (-1)^|alpha| / alpha! D_{alpha + e_q}(R) M_alpha,
 * which takes the derivative tensor one order above the multipoles'; ix1 is
 * the index of order ix->p + 1 (its first ix->nc entries are ix's). */
static void or_m2p_grad(const or_index* ix, const or_index* ix1, const double* M, const double R[3], double g[3]) {
  double D[1000];
  or_dtensor_ix(ix1, R, ix1->p, D);
  g[0] = g[1] = g[2] = 0.0;
  for (int ka = 0; ka < ix->nc; ++ka) {
    const int* a = ix->mi[ka];
    const int na = a[0] + a[1] + a[2];
    if (na > ix->mo) continue;
    const double w = ((na & 1) ? -1.0 : 1.0) / (or_fact(a[0]) * or_fact(a[1]) * or_fact(a[2])) * M[ka];
    for (int q = 0; q < 3; ++q)
#if ORACLE_MUTANT == 18 /* planted mistake: the gradient reads D_alpha instead of D_{alpha + e_q} */
      g[q] += w * D[ix1->lut[a[0]][a[1]][a[2]]];
#else
      g[q] += w * D[ix1->lut[a[0] + (q == 0)][a[1] + (q == 1)][a[2] + (q == 2)]];
#endif
  }
}

/* M2P of one multipole set at one point, with its gradient (test hook for
 * the pins of or_m2p_grad). */
int oracle_m2p_eval(const double* M, int p, const double* R, double* phi, double* grad) {
  if (p < 0 || p + 1 > OR_MAXP) return -1;
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index* ix1 = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  or_index_init(ix1, p + 1);
  *phi = or_m2p(ix, M, R);
  or_m2p_grad(ix, ix1, M, R, grad);
  free(ix);
  free(ix1);
  return 0;
}

/* Analytic acceleration with either final stage (final_stage 0: the leaf
 * M2L and L2P, as oracle_fmm_accel; 1: the leaf locals are the parent's
 * shifted locals alone and the leaf interaction list is evaluated by M2P at
 * the cell centre, Sec. 4):
 *   accel = -G dx ( grad L2P(L_leaf) [+ sum_{S in IL} grad M2P(M_S)]
 *                   + sum_near m (x - y) / |x - y|^3 ). */
int oracle_fmm_accel_ex(const double* rho, int nx, int ny, int nz, int b, int p, int final_stage, double dx, double G,
                        double* accel, int nthreads) {
  or_hier H;
  if (or_hier_init(&H, nx, ny, nz, b, p)) return -1;
  if (final_stage < 0 || final_stage > 1 || p + 1 > OR_MAXP) return -1;
  or_set_threads(nthreads);
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index* ix1 = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  or_index_init(ix1, p + 1);
  double** M = or_upward(&H, ix, rho);
  double** L = or_downward_ex(&H, ix, M, final_stage ? 0 : 1);
  const long n = (long)nx * ny * nz;
  const double scale = -G * dx;
  const or_level* lf = &H.lev[H.L];
#pragma omp parallel for schedule(dynamic, 64)
  for (long c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    double gf[3], gn[3];
    or_far_grad(&H, ix, L, x, y, z, gf);
    if (final_stage && H.L >= 2) {
      int il[216][3];
      const int m = or_ilist(&H, H.L, x / b, y / b, z / b, il);
      for (int q = 0; q < m; ++q) {
        double cs[3], g[3];
        or_bcentre(lf, il[q][0], il[q][1], il[q][2], cs);
        const double R[3] = {x + 0.5 - cs[0], y + 0.5 - cs[1], z + 0.5 - cs[2]};
        or_m2p_grad(ix, ix1, M[H.L] + or_bidx(lf, il[q][0], il[q][1], il[q][2]) * ix->nc, R, g);
        for (int r = 0; r < 3; ++r) gf[r] += g[r];
      }
    }
    or_near_grad(&H, rho, x, y, z, gn);
    for (int q = 0; q < 3; ++q) accel[q * n + c] = scale * (gf[q] + gn[q]);
  }
  or_free_levels(&H, M);
  or_free_levels(&H, L);
  free(ix);
  free(ix1);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Analytic acceleration (the force read off the expansions and the near    */
/* pair forces, instead of the stencil of App. C):                          */
/*   accel = -G dx ( grad L2P(L_leaf) + sum_near m (x - y) / |x - y|^3 )    */
/* in cell units for the gradients (physical accel = -grad_phys phi).       */
/* ------------------------------------------------------------------------ */

int oracle_fmm_accel(const double* rho, int nx, int ny, int nz, int b, int p, double dx, double G, double* accel,
                     int nthreads) {
  or_hier H;
  if (or_hier_init(&H, nx, ny, nz, b, p)) return -1;
  or_set_threads(nthreads);
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  double** M = or_upward(&H, ix, rho);
  double** L = or_downward(&H, ix, M);
  const long n = (long)nx * ny * nz;
  const double scale = -G * dx;
#pragma omp parallel for schedule(dynamic, 64)
  for (long c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    double gf[3], gn[3];
    or_far_grad(&H, ix, L, x, y, z, gf);
    or_near_grad(&H, rho, x, y, z, gn);
    for (int q = 0; q < 3; ++q) accel[q * n + c] = scale * (gf[q] + gn[q]);
  }
  or_free_levels(&H, M);
  or_free_levels(&H, L);
  free(ix);
  return 0;
}

/* O(N^2) pair forces: accel(x) = -G dx sum_{y != x} m_y (x - y) / |x - y|^3. */
int oracle_direct_accel(const double* rho, int nx, int ny, int nz, double dx, double G, double* accel, int nthreads) {
  or_set_threads(nthreads);
  const long n = (long)nx * ny * nz;
  const double scale = -G * dx;
#pragma omp parallel for schedule(dynamic, 16)
  for (long c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    double s[3] = {0.0, 0.0, 0.0};
    for (long d = 0; d < n; ++d) {
      double m = rho[d];
      if (m == 0.0) continue;
      int sx = (int)(d % nx), sy = (int)((d / nx) % ny), sz = (int)(d / ((long)nx * ny));
      double g[3];
      or_grad_g((double)(x - sx), (double)(y - sy), (double)(z - sz), g);
      for (int q = 0; q < 3; ++q) s[q] += m * g[q];
    }
    for (int q = 0; q < 3; ++q) accel[q * n + c] = scale * s[q];
  }
  return 0;
}

/* Analytic acceleration at a sample of cells (any grid size): ancestor chain
 * of local expansions as oracle_fmm_sample, then the gradients. */
int oracle_fmm_sample_accel(const double* rho, int nx, int ny, int nz, int b, int p, double dx, double G,
                            long nsample, const long* cells, double* accel_out /* [nsample][3] */, int nthreads) {
  or_hier H;
  if (or_hier_init(&H, nx, ny, nz, b, p)) return -1;
  or_set_threads(nthreads);
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  double** M = or_upward(&H, ix, rho);
  const double scale = -G * dx;
  const or_level* lf = &H.lev[H.L];
#pragma omp parallel for schedule(dynamic, 1)
  for (long s = 0; s < nsample; ++s) {
    long c = cells[s];
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    int bi = x / H.b, bj = y / H.b, bk = z / H.b;
    double* Lb = (double*)malloc(sizeof(double) * ix->nc);
    or_local_chain(&H, ix, M, H.L, bi, bj, bk, Lb);
    double cc[3];
    or_bcentre(lf, bi, bj, bk, cc);
    double e[3] = {x + 0.5 - cc[0], y + 0.5 - cc[1], z + 0.5 - cc[2]};
    double gf[3], gn[3];
    or_l2p_grad(ix, Lb, e, gf);
    free(Lb);
    or_near_grad(&H, rho, x, y, z, gn);
    for (int q = 0; q < 3; ++q) accel_out[3 * s + q] = scale * (gf[q] + gn[q]);
  }
  or_free_levels(&H, M);
  free(ix);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* The paper's own final stage (Sec. 4): at the leaf level the interaction  */
/* list is evaluated by M2P at the cell centres instead of M2L + L2P:       */
/*   phi(x) = L2P(L2L(L_parent)) + sum_{S in IL(B)} M2P(M_S, x - c_S)      */
/*            + near(x)                                                     */
/* ------------------------------------------------------------------------ */

/* Potential with separate order limits: multipoles to order mo and locals to
 * order lo inside |alpha| + |beta| <= p (the paper keeps multipoles to order
 * 2 and locals to order 3, Sec. 2.1 and 2.3), final stage M2L + L2P
 * (final_stage = 0) or M2P at the cell centres (1, Sec. 4).  Multipole
 * components above mo and local components above lo take no part: M2L and
 * M2P skip them, so L2L and L2P see zeros there.  mo = lo = p gives
 * oracle_fmm's potential (final_stage 0) and oracle_fmm_m2p's (1). */
int oracle_fmm_orders(const double* rho, int nx, int ny, int nz, int b, int p, int mo, int lo, int final_stage,
                      double dx, double G, double* phi, int nthreads) {
  or_hier H;
  if (or_hier_init(&H, nx, ny, nz, b, p)) return -1;
  if (mo < 0 || mo > p || lo < 0 || lo > p || final_stage < 0 || final_stage > 1) return -1;
  or_set_threads(nthreads);
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  or_index_init(ix, p);
  ix->mo = mo;
  ix->lo = lo;
  double** M = or_upward(&H, ix, rho);
  double** L = or_downward_ex(&H, ix, M, final_stage ? 0 : 1);
  const long n = (long)nx * ny * nz;
  const double scale = G * dx * dx;
  const or_level* lf = &H.lev[H.L];
#pragma omp parallel for schedule(dynamic, 64)
  for (long c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
    double s = or_far_cell(&H, ix, L, x, y, z);
    if (final_stage && H.L >= 2) {
      int il[216][3];
      int m = or_ilist(&H, H.L, x / b, y / b, z / b, il);
      for (int q = 0; q < m; ++q) {
        double cs[3];
        or_bcentre(lf, il[q][0], il[q][1], il[q][2], cs);
        double R[3] = {x + 0.5 - cs[0], y + 0.5 - cs[1], z + 0.5 - cs[2]};
        s += or_m2p(ix, M[H.L] + or_bidx(lf, il[q][0], il[q][1], il[q][2]) * ix->nc, R);
      }
    }
    s += or_near_cell(&H, rho, x, y, z);
    phi[c] = scale * s;
  }
  or_free_levels(&H, M);
  or_free_levels(&H, L);
  free(ix);
  return 0;
}

int oracle_fmm_m2p(const double* rho, int nx, int ny, int nz, int b, int p, double dx, double G, double* phi,
                   int nthreads) {
  return oracle_fmm_orders(rho, nx, ny, nz, b, p, p, p, 1, dx, G, phi, nthreads);
}
