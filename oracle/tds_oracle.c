/*
 * tds_oracle.c -- plain FP64 CPU oracle for one time step of the active-soil
 * particle system (see tds_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path. It shares no code
 * with the CUDA library. Compile with -ffp-contract=off: the contact
 * predicate is part of a bit-exact contract with the GPU path.
 *
 * Paper sections followed (Servin, Berglund, Nystedt, "A multiscale model of
 * terrain dynamics for real-time earthmoving simulation"):
 *   - contact law, Eqs. signCoul1-3 (normal complementarity with cohesion
 *     bound f_c, Coulomb friction disk, rolling-resistance ball);
 *   - Hertz mapping k_n = E* sqrt(d*)/3, g_n = delta^{5/4}, eps_n = 5/(4 k_n),
 *     and tau_n = 2 dt for resting contacts;
 *   - SPOOK: p = M v_n + dt f, q = -(4/dt) Upsilon g + Upsilon G v_n,
 *     Sigma = (4/dt^2) eps Upsilon, Sigma_bar = gamma/dt,
 *     Upsilon = 1/(1 + 4 tau/dt), x_{n+1} = x_n + dt v_{n+1};
 *   - Algorithm 1: collision detection, iterative PGS, position update;
 *   - Eq. eqmotb: particles feel gravity, tool, terrain and particle contacts.
 *
 * Readings taken where the paper is silent, garbled or inconsistent:
 *   R1 g_n is printed as delta^{5/4} but must be >= 0 without penetration:
 *      read g_n = -delta^{5/4} (delta = overlap).
 *   R2 "eps_n = 5/4 k_n" is read as 5/(4 k_n) (units; potential (2/5)k delta^{5/2}).
 *   R3 Unit-Jacobian form: dividing the row G v + Sigma lambda = q by
 *      s = |G_n| = (5/4) delta^{1/4} gives, for the physical impulse
 *      Lambda = s lambda, J v + Sigma_eff Lambda = q_eff with
 *      Sigma_eff = (4/dt^2) Upsilon 4/(5 k_n sqrt(delta)) and
 *      g_eff = -(4/5) delta. Equilibrium: k_n delta^{3/2} = load (Hertz).
 *      sqrt(delta) is floored at delta_floor = 1e-5 (r_a + r_b).
 *   R4 lambda is an impulse; f_c = c_p A_p / |G_n^T| is a force, so the bound
 *      on the physical impulse is dt c_p pi rbar^2.
 *   R5 Cohesive overlap "delta_c = 0.025 d": contacts exist while the gap is
 *      below delta_c = 0.025 (r_a + r_b) (static: 0.025 * 2 r_a) when c_p > 0,
 *      and the cohesion bound acts there. Tool contacts have no cohesion.
 *   R6 Friction bound mu_t |Lambda_n| (the literal |G_n^T lambda_n|), so
 *      cohesive tension also gives friction.
 *   R7 Rolling radius of a pair: harmonic mean rbar = 2 r_a r_b/(r_a + r_b)
 *      (equals r for equal spheres); static: r_a. A_p = pi rbar^2.
 *   R8 Friction is a disk, rolling resistance a 3-D ball (6 rows per contact).
 *   R9 gamma_t = gamma_r = 1e-9 (paper silent), relaxation 1.
 *   R10 The heightfield is triangulated with the diagonal from (i+1,j) to
 *      (i,j+1); one heightfield contact per particle.
 *   R11 Static surfaces are rigid: E* = E/(1 - nu^2), d* = d_a.
 *   R12 The velocity coefficient of q is the printed Upsilon (not 4 tau/dt Upsilon).
 *   R13 A kinematic tool contributes its point velocity v_T + w_T x (x_c - p_T)
 *      to the normal and tangent rows and w_T to the rolling row.
 */
#include "tds_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* FP64 vector helpers                                                 */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double a[3], const double b[3], double o[3]) {
  double t0 = a[1] * b[2] - a[2] * b[1];
  double t1 = a[2] * b[0] - a[0] * b[2];
  double t2 = a[0] * b[1] - a[1] * b[0];
  o[0] = t0; o[1] = t1; o[2] = t2;
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------------------------ */
/* Box geometry contract: quaternion -> matrix and tool-frame            */
/* composition are evaluated in FP64 in exactly this order and rounded   */
/* to FP32; the FP32 predicate then reads the rounded values.            */
/* ------------------------------------------------------------------ */
static void quat_matrix(const float qf[4], double R[9]) {
  double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
  double s = 1.0 / sqrt(((w * w + x * x) + y * y) + z * z);
  w *= s; x *= s; y *= s; z *= s;
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - w * z);
  R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);
  R[7] = 2.0 * (y * z + w * x);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
}

typedef struct {
  float c[3], R[9], h[3]; /* world frame, FP32 */
  int is_tool;
} wbox;

/* World-frame boxes: the walls first, then the tool boxes. */
static wbox *world_boxes(const orc_params *P, int *nb) {
  int n = P->n_walls + P->n_tool;
  *nb = n;
  wbox *B = (wbox *)calloc(n > 0 ? n : 1, sizeof(wbox));
  if (!B) return NULL;
  for (int k = 0; k < P->n_walls; ++k) {
    const float *d = P->walls + 10 * k;
    double R[9];
    quat_matrix(d + 3, R);
    for (int i = 0; i < 3; ++i) { B[k].c[i] = d[i]; B[k].h[i] = d[7 + i]; }
    for (int i = 0; i < 9; ++i) B[k].R[i] = (float)R[i];
    B[k].is_tool = 0;
  }
  double RT[9];
  quat_matrix(P->tool_quat, RT);
  for (int k = 0; k < P->n_tool; ++k) {
    const float *d = P->tool_boxes + 10 * k;
    double Rk[9], Rw[9];
    quat_matrix(d + 3, Rk);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        Rw[3 * i + j] = (RT[3 * i + 0] * Rk[0 + j] + RT[3 * i + 1] * Rk[3 + j]) +
                        RT[3 * i + 2] * Rk[6 + j];
    wbox *b = &B[P->n_walls + k];
    for (int i = 0; i < 3; ++i) {
      double off = (RT[3 * i + 0] * (double)d[0] + RT[3 * i + 1] * (double)d[1]) +
                   RT[3 * i + 2] * (double)d[2];
      b->c[i] = (float)((double)P->tool_pos[i] + off);
      b->h[i] = d[7 + i];
    }
    for (int i = 0; i < 9; ++i) b->R[i] = (float)Rw[i];
    b->is_tool = 1;
  }
  return B;
}

/* ------------------------------------------------------------------ */
/* FP32 contact predicates (bit-exact contract; -ffp-contract=off)      */
/* ------------------------------------------------------------------ */
static int pp_touch(float xa, float ya, float za, float ra, float xb, float yb,
                    float zb, float rb, int cohesive) {
  float dx = xb - xa, dy = yb - ya, dz = zb - za;
  float d2 = (dx * dx + dy * dy) + dz * dz;
  float rs = ra + rb;
  float R = cohesive ? rs + 0.025f * rs : rs;
  return d2 < R * R;
}

static float static_reach(float r, int cohesive) {
  return cohesive ? r + 0.025f * (r + r) : r;
}

/* Triangle of the heightfield under (px, py); returns the FP32 signed
 * distance from the triangle's plane and the triangle description. */
typedef struct { int i, j, upper; } hf_tri;

static float hf_signed_distance(const orc_params *P, float px, float py, float pz,
                                hf_tri *t) {
  int nx = P->hf_nx, ny = P->hf_ny, stride = nx + 1;
  float tx = (px - P->hf_x0) / P->hf_cell;
  float ty = (py - P->hf_y0) / P->hf_cell;
  float fx = floorf(tx), fy = floorf(ty);
  int i, j;
  if (!(fx >= 0.0f)) i = 0; else if (fx > (float)(nx - 1)) i = nx - 1; else i = (int)fx;
  if (!(fy >= 0.0f)) j = 0; else if (fy > (float)(ny - 1)) j = ny - 1; else j = (int)fy;
  float u = tx - (float)i, v = ty - (float)j;
  const float *h = P->hf_h;
  float hb, a, b, uu, vv;
  int upper = !(u + v <= 1.0f);
  if (!upper) {
    hb = h[j * stride + i];
    a = h[j * stride + i + 1] - hb;
    b = h[(j + 1) * stride + i] - hb;
    uu = u; vv = v;
  } else {
    hb = h[(j + 1) * stride + i + 1];
    a = h[(j + 1) * stride + i] - hb;
    b = h[j * stride + i + 1] - hb;
    uu = 1.0f - u; vv = 1.0f - v;
  }
  float e = pz - hb;
  e = e - a * uu;
  e = e - b * vv;
  float num = P->hf_cell * e;
  float den = sqrtf((P->hf_cell * P->hf_cell + a * a) + b * b);
  t->i = i; t->j = j; t->upper = upper;
  return num / den;
}

static int box_touch(const wbox *B, float px, float py, float pz, float reach) {
  float dx = px - B->c[0], dy = py - B->c[1], dz = pz - B->c[2];
  float l[3], e[3];
  for (int k = 0; k < 3; ++k) {
    l[k] = (B->R[k] * dx + B->R[3 + k] * dy) + B->R[6 + k] * dz;
    float q = fminf(fmaxf(l[k], -B->h[k]), B->h[k]);
    e[k] = l[k] - q;
  }
  float d2 = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2];
  return d2 < reach * reach;
}

/* ------------------------------------------------------------------ */
/* Contact detection                                                    */
/* ------------------------------------------------------------------ */
typedef struct { int64_t cell; int idx; } cell_entry;

static int cmp_cell(const void *pa, const void *pb) {
  const cell_entry *a = (const cell_entry *)pa, *b = (const cell_entry *)pb;
  if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
  return a->idx - b->idx;
}
static int cmp_u64(const void *pa, const void *pb) {
  uint64_t a = *(const uint64_t *)pa, b = *(const uint64_t *)pb;
  return a < b ? -1 : (a > b ? 1 : 0);
}

typedef struct { uint64_t *k; int n, cap, overflow; } keylist;
static void kl_push(keylist *L, uint64_t key) {
  if (L->n < L->cap) L->k[L->n] = key;
  else L->overflow = 1;
  L->n++;
}

/* Appends every contact key (unsorted). */
static int detect(const orc_params *P, int n, const double *x, const double *r,
                  int brute, const wbox *B, int nb, keylist *L) {
  int cohesive = P->cohesion > 0.0;
  float *xf = (float *)malloc(sizeof(float) * 4 * (n > 0 ? n : 1));
  if (!xf) return -2;
  double rmax = 0.0;
  for (int i = 0; i < n; ++i) {
    xf[4 * i + 0] = (float)x[3 * i + 0];
    xf[4 * i + 1] = (float)x[3 * i + 1];
    xf[4 * i + 2] = (float)x[3 * i + 2];
    xf[4 * i + 3] = (float)r[i];
    if (r[i] > rmax) rmax = r[i];
  }
  /* particle-particle (radius 0: a dormant reserve slot, never in contact) */
  if (brute) {
    for (int a = 0; a < n; ++a)
      for (int b = a + 1; b < n; ++b)
        if (r[a] > 0.0 && r[b] > 0.0 && pp_touch(xf[4 * a], xf[4 * a + 1], xf[4 * a + 2], xf[4 * a + 3], xf[4 * b],
                     xf[4 * b + 1], xf[4 * b + 2], xf[4 * b + 3], cohesive))
          kl_push(L, ((uint64_t)a << 32) | (uint64_t)b);
  } else if (n > 0) {
    /* uniform grid of cells wider than any contact reach; neighbours are
     * found in the 27 surrounding cells, and the predicate decides. */
    double cell = 2.1 * rmax;
    if (!(cell > 0.0)) cell = 1.0;
    double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < 3; ++k) {
        if (!(r[i] > 0.0)) continue;
        if (x[3 * i + k] < lo[k]) lo[k] = x[3 * i + k];
        if (x[3 * i + k] > hi[k]) hi[k] = x[3 * i + k];
      }
    if (!(lo[0] <= hi[0])) for (int k = 0; k < 3; ++k) lo[k] = hi[k] = 0.0;
    int64_t dim[3];
    for (int k = 0; k < 3; ++k) dim[k] = (int64_t)floor((hi[k] - lo[k]) / cell) + 3;
    cell_entry *E = (cell_entry *)malloc(sizeof(cell_entry) * n);
    if (!E) { free(xf); return -2; }
    int64_t (*ci)[3] = malloc(sizeof(int64_t[3]) * n);
    if (!ci) { free(E); free(xf); return -2; }
    int na = 0;  /* active particles in E */
    for (int i = 0; i < n; ++i) {
      if (!(r[i] > 0.0)) continue;
      for (int k = 0; k < 3; ++k) ci[i][k] = (int64_t)floor((x[3 * i + k] - lo[k]) / cell) + 1;
      E[na].cell = (ci[i][2] * dim[1] + ci[i][1]) * dim[0] + ci[i][0];
      E[na].idx = i;
      ++na;
    }
    qsort(E, na, sizeof(cell_entry), cmp_cell);
    for (int a = 0; a < n; ++a) {
      if (!(r[a] > 0.0)) continue;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int64_t c = ((ci[a][2] + dz) * dim[1] + (ci[a][1] + dy)) * dim[0] + ci[a][0] + dx;
            /* lower bound of cell c */
            int lo_i = 0, hi_i = na;
            while (lo_i < hi_i) {
              int mid = (lo_i + hi_i) / 2;
              if (E[mid].cell < c) lo_i = mid + 1; else hi_i = mid;
            }
            for (int m = lo_i; m < na && E[m].cell == c; ++m) {
              int b = E[m].idx;
              if (b <= a) continue;
              if (pp_touch(xf[4 * a], xf[4 * a + 1], xf[4 * a + 2], xf[4 * a + 3], xf[4 * b],
                           xf[4 * b + 1], xf[4 * b + 2], xf[4 * b + 3], cohesive))
                kl_push(L, ((uint64_t)a << 32) | (uint64_t)b);
            }
          }
    }
    free(ci);
    free(E);
  }
  /* particle-heightfield and particle-box */
  for (int a = 0; a < n; ++a) {
    float px = xf[4 * a], py = xf[4 * a + 1], pz = xf[4 * a + 2], ra = xf[4 * a + 3];
    if (!(r[a] > 0.0)) continue;
    if (P->hf_nx > 0) {
      hf_tri t;
      float s = hf_signed_distance(P, px, py, pz, &t);
      if (s < static_reach(ra, cohesive))
        kl_push(L, ((uint64_t)a << 32) | ORC_STATIC_BIT | 0u);
    }
    for (int k = 0; k < nb; ++k) {
      float reach = static_reach(ra, cohesive && !B[k].is_tool);
      if (box_touch(&B[k], px, py, pz, reach))
        kl_push(L, ((uint64_t)a << 32) | ORC_STATIC_BIT | (uint64_t)(1 + k));
    }
  }
  free(xf);
  return 0;
}

int32_t orc_find_contacts(const orc_params *P, int32_t n, const double *x,
                          const double *r, int32_t brute, int32_t cap,
                          uint64_t *keys) {
  if (!P || n < 0 || (n > 0 && (!x || !r)) || cap < 0) return -2;
  int nb;
  wbox *B = world_boxes(P, &nb);
  if (!B) return -2;
  keylist L = {keys, 0, cap, 0};
  int rc = detect(P, n, x, r, brute, B, nb, &L);
  free(B);
  if (rc) return rc;
  if (L.overflow) return -1;
  qsort(keys, L.n, sizeof(uint64_t), cmp_u64);
  return L.n;
}

/* ------------------------------------------------------------------ */
/* Colouring priority: SplitMix64 output function (Steele, Lea, Flood,  */
/* OOPSLA 2014), a bijection on 64-bit words.                           */
/* ------------------------------------------------------------------ */
uint64_t orc_priority(uint64_t key) {
  uint64_t z = key + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* ------------------------------------------------------------------ */
/* Contacts with their rows                                             */
/* ------------------------------------------------------------------ */
typedef struct {
  uint64_t key, prio;
  int a, b;          /* b < 0: static surface */
  int surf, is_tool;
  double n[3];       /* unit normal from a towards b (into the static surface) */
  double delta;      /* overlap */
  double la, lb;     /* lever arms from the centres to the contact point */
  double xc[3];      /* contact point */
  double t1[3], t2[3];
  double vs[3], ws[3];            /* static surface point velocity, spin */
  double Sn, qn, fc, mu, rmu;     /* normal row and bounds */
  double Dn, Dt, Dr;              /* diagonal of G M^-1 G^T + Sigma per row group */
  double st, sr;                  /* Sigma_bar of the tangent and rolling rows */
  double ln, lt[2], lr[3];        /* impulses */
  double Gvn;                     /* G_n v_n at the start of the step */
  int colour;
  int kept_colour;                /* incremental colouring: the previous step's colour, or -1 */
  int persisted;                  /* the key existed in the previous step */
  double W;                       /* impulse scale m_eff |g| h of the learned warm start */
  double sdir[3];                 /* slip direction s of the learned warm start */
  double feat[10];
} contact;

typedef struct {
  double *m_inv, *I_inv; /* per particle */
} masses;

static void tangent_basis(const double n[3], double t1[3], double t2[3]) {
  /* the axis least aligned with n (ties: lowest index) */
  int k = 0;
  double best = fabs(n[0]);
  if (fabs(n[1]) < best) { best = fabs(n[1]); k = 1; }
  if (fabs(n[2]) < best) { k = 2; }
  double e[3] = {0.0, 0.0, 0.0};
  e[k] = 1.0;
  cross3(n, e, t1);
  double s = norm3(t1);
  t1[0] /= s; t1[1] /= s; t1[2] /= s;
  cross3(n, t1, t2);
}

/* Geometry (FP64) of a contact whose existence the FP32 predicate decided. */
static void contact_geometry(const orc_params *P, const wbox *B, const double *x,
                             const double *r, contact *c) {
  const double *xa = x + 3 * c->a;
  double ra = r[c->a];
  if (c->b >= 0) {
    const double *xb = x + 3 * c->b;
    double d[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
    double dist = norm3(d);
    if (dist > 0.0) { c->n[0] = d[0] / dist; c->n[1] = d[1] / dist; c->n[2] = d[2] / dist; }
    else { c->n[0] = 0.0; c->n[1] = 0.0; c->n[2] = 1.0; }
    c->delta = ra + r[c->b] - dist;
    c->la = ra - 0.5 * c->delta;
    c->lb = r[c->b] - 0.5 * c->delta;
  } else {
    double s, ns[3];
    if (c->surf == 0) {
      hf_tri t;
      (void)hf_signed_distance(P, (float)xa[0], (float)xa[1], (float)xa[2], &t);
      int stride = P->hf_nx + 1;
      const float *h = P->hf_h;
      double cell = P->hf_cell;
      double u = (xa[0] - (double)P->hf_x0) / cell - t.i;
      double v = (xa[1] - (double)P->hf_y0) / cell - t.j;
      double hb, a, b, uu, vv;
      if (!t.upper) {
        hb = h[t.j * stride + t.i];
        a = h[t.j * stride + t.i + 1] - hb;
        b = h[(t.j + 1) * stride + t.i] - hb;
        uu = u; vv = v;
      } else {
        hb = h[(t.j + 1) * stride + t.i + 1];
        a = h[(t.j + 1) * stride + t.i] - hb;
        b = h[t.j * stride + t.i + 1] - hb;
        uu = 1.0 - u; vv = 1.0 - v;
      }
      double den = sqrt(cell * cell + a * a + b * b);
      s = cell * (xa[2] - hb - a * uu - b * vv) / den;
      if (!t.upper) { ns[0] = -a / den; ns[1] = -b / den; }
      else { ns[0] = a / den; ns[1] = b / den; }
      ns[2] = cell / den;
    } else {
      const wbox *bx = &B[c->surf - 1];
      double R[9], cc[3], hh[3], l[3], e[3];
      for (int i = 0; i < 9; ++i) R[i] = bx->R[i];
      for (int i = 0; i < 3; ++i) { cc[i] = bx->c[i]; hh[i] = bx->h[i]; }
      double d[3] = {xa[0] - cc[0], xa[1] - cc[1], xa[2] - cc[2]};
      int inside = 1;
      for (int k = 0; k < 3; ++k) {
        l[k] = R[k] * d[0] + R[3 + k] * d[1] + R[6 + k] * d[2];
        double q = l[k] < -hh[k] ? -hh[k] : (l[k] > hh[k] ? hh[k] : l[k]);
        e[k] = l[k] - q;
        if (e[k] != 0.0) inside = 0;
      }
      if (!inside) {
        s = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        for (int i = 0; i < 3; ++i)
          ns[i] = (R[3 * i + 0] * e[0] + R[3 * i + 1] * e[1] + R[3 * i + 2] * e[2]) / s;
      } else {
        int k = 0;
        double depth = hh[0] - fabs(l[0]);
        for (int m = 1; m < 3; ++m)
          if (hh[m] - fabs(l[m]) < depth) { depth = hh[m] - fabs(l[m]); k = m; }
        double side = l[k] >= 0.0 ? 1.0 : -1.0;
        s = -depth;
        for (int i = 0; i < 3; ++i) ns[i] = side * R[3 * i + k];
      }
    }
    c->n[0] = -ns[0]; c->n[1] = -ns[1]; c->n[2] = -ns[2];
    c->delta = ra - s;
    c->la = ra - 0.5 * c->delta;
    c->lb = 0.0;
  }
  for (int i = 0; i < 3; ++i) c->xc[i] = xa[i] + c->la * c->n[i];
  tangent_basis(c->n, c->t1, c->t2);
  for (int i = 0; i < 3; ++i) { c->vs[i] = 0.0; c->ws[i] = 0.0; }
  if (c->is_tool) {
    double rel[3] = {c->xc[0] - P->tool_pos[0], c->xc[1] - P->tool_pos[1],
                     c->xc[2] - P->tool_pos[2]};
    double wT[3] = {P->tool_angvel[0], P->tool_angvel[1], P->tool_angvel[2]};
    double wxr[3];
    cross3(wT, rel, wxr);
    for (int i = 0; i < 3; ++i) { c->vs[i] = P->tool_vel[i] + wxr[i]; c->ws[i] = wT[i]; }
  }
}

/* Row coefficients of the contact law with the Hertz mapping and SPOOK. */
static void contact_rows(const orc_params *P, const double *r, const masses *M,
                         const double *v0, contact *c) {
  double h = P->dt;
  double nu = P->poisson, E = P->young;
  double ra = r[c->a];
  double Estar, dstar, rbar, dfloor, ima = M->m_inv[c->a], iIa = M->I_inv[c->a];
  double imb = 0.0, iIb = 0.0;
  double vb[3];
  if (c->b >= 0) {
    double rb = r[c->b];
    Estar = 1.0 / (2.0 * (1.0 - nu * nu) / E);
    dstar = 1.0 / (1.0 / (2.0 * ra) + 1.0 / (2.0 * rb));
    rbar = 2.0 * ra * rb / (ra + rb);
    dfloor = 1e-5 * (ra + rb);
    imb = M->m_inv[c->b]; iIb = M->I_inv[c->b];
    for (int i = 0; i < 3; ++i) vb[i] = v0[3 * c->b + i];
  } else {
    Estar = E / (1.0 - nu * nu);
    dstar = 2.0 * ra;
    rbar = ra;
    dfloor = 1e-5 * 2.0 * ra;
    for (int i = 0; i < 3; ++i) vb[i] = c->vs[i];
  }
  double kn = Estar * sqrt(dstar) / 3.0;
  double ds = c->delta > dfloor ? c->delta : dfloor;
  double eps = 4.0 / (5.0 * kn * sqrt(ds));
  double tau = 2.0 * h;
  double ups = 1.0 / (1.0 + 4.0 * tau / h);
  double g = -0.8 * c->delta;
  double dv[3] = {vb[0] - v0[3 * c->a], vb[1] - v0[3 * c->a + 1], vb[2] - v0[3 * c->a + 2]};
  double Gv0 = dot3(c->n, dv);
  c->Gvn = Gv0;
  c->Sn = 4.0 / (h * h) * ups * eps;
  c->qn = -4.0 / h * ups * g + ups * Gv0;
  c->fc = (P->cohesion > 0.0 && !c->is_tool) ? h * P->cohesion * ORC_PI * rbar * rbar : 0.0;
  c->mu = c->is_tool ? P->mu_tool : P->mu_t;
  c->rmu = rbar * P->mu_r;
  c->st = P->gamma_t / h;
  c->sr = P->gamma_r / h;
  c->Dn = ima + imb + c->Sn;
  c->Dt = ima + imb + c->la * c->la * iIa + c->lb * c->lb * iIb + c->st;
  c->Dr = iIa + iIb + c->sr;
}

/* Apply the impulse increment (dn along n, dt world tangent, dr rolling). */
static void apply(const contact *c, const masses *M, double *v, double *w, double dn,
                  const double dt[3], const double dr[3]) {
  double P[3] = {dn * c->n[0] + dt[0], dn * c->n[1] + dt[1], dn * c->n[2] + dt[2]};
  double ima = M->m_inv[c->a], iIa = M->I_inv[c->a];
  double ra_arm[3] = {c->la * c->n[0], c->la * c->n[1], c->la * c->n[2]};
  double ta[3];
  cross3(ra_arm, dt, ta);
  for (int i = 0; i < 3; ++i) {
    v[3 * c->a + i] -= ima * P[i];
    w[3 * c->a + i] -= iIa * (ta[i] + dr[i]);
  }
  if (c->b >= 0) {
    double imb = M->m_inv[c->b], iIb = M->I_inv[c->b];
    double rb_arm[3] = {-c->lb * c->n[0], -c->lb * c->n[1], -c->lb * c->n[2]};
    double tb[3];
    cross3(rb_arm, dt, tb);
    for (int i = 0; i < 3; ++i) {
      v[3 * c->b + i] += imb * P[i];
      w[3 * c->b + i] += iIb * (tb[i] + dr[i]);
    }
  }
}

/* Velocities of the two sides. */
static void side_velocities(const contact *c, const double *v, const double *w,
                            double va[3], double wa[3], double vb[3], double wb[3]) {
  for (int i = 0; i < 3; ++i) { va[i] = v[3 * c->a + i]; wa[i] = w[3 * c->a + i]; }
  if (c->b >= 0)
    for (int i = 0; i < 3; ++i) { vb[i] = v[3 * c->b + i]; wb[i] = w[3 * c->b + i]; }
  else
    for (int i = 0; i < 3; ++i) { vb[i] = c->vs[i]; wb[i] = c->ws[i]; }
}

/* Relative velocity of the contact points: (v_b + w_b x (-lb n)) - (v_a + w_a x (la n)) */
static void slip_velocity(const contact *c, const double va[3], const double wa[3],
                          const double vb[3], const double wb[3], double u[3]) {
  double arm_a[3] = {c->la * c->n[0], c->la * c->n[1], c->la * c->n[2]};
  double arm_b[3] = {-c->lb * c->n[0], -c->lb * c->n[1], -c->lb * c->n[2]};
  double xa[3], xb[3];
  cross3(wa, arm_a, xa);
  cross3(wb, arm_b, xb);
  for (int i = 0; i < 3; ++i) u[i] = (vb[i] + xb[i]) - (va[i] + xa[i]);
}

static void project_ball(double *y, int dim, double bound) {
  double s = 0.0;
  for (int i = 0; i < dim; ++i) s += y[i] * y[i];
  s = sqrt(s);
  if (s > bound) {
    double f = bound > 0.0 ? bound / s : 0.0;
    for (int i = 0; i < dim; ++i) y[i] *= f;
  }
}

/* One projected Gauss-Seidel update of one contact: normal row, then the
 * 2-D tangent rows (Coulomb disk), then the 3 rolling rows (ball), each
 * followed by v += M^-1 G^T dLambda. */
static void pgs_contact(contact *c, const masses *M, double *v, double *w) {
  double va[3], wa[3], vb[3], wb[3], zero[3] = {0.0, 0.0, 0.0};
  /* normal */
  side_velocities(c, v, w, va, wa, vb, wb);
  double dv[3] = {vb[0] - va[0], vb[1] - va[1], vb[2] - va[2]};
  double res = dot3(c->n, dv) + c->Sn * c->ln - c->qn;
  double ln = c->ln - res / c->Dn;
  if (ln < -c->fc) ln = -c->fc;
  double dln = ln - c->ln;
  c->ln = ln;
  apply(c, M, v, w, dln, zero, zero);
  /* tangent */
  side_velocities(c, v, w, va, wa, vb, wb);
  double u[3];
  slip_velocity(c, va, wa, vb, wb, u);
  double y[2];
  y[0] = c->lt[0] - (dot3(c->t1, u) + c->st * c->lt[0]) / c->Dt;
  y[1] = c->lt[1] - (dot3(c->t2, u) + c->st * c->lt[1]) / c->Dt;
  project_ball(y, 2, c->mu * fabs(c->ln));
  double d0 = y[0] - c->lt[0], d1 = y[1] - c->lt[1];
  c->lt[0] = y[0]; c->lt[1] = y[1];
  double dtw[3] = {d0 * c->t1[0] + d1 * c->t2[0], d0 * c->t1[1] + d1 * c->t2[1],
                   d0 * c->t1[2] + d1 * c->t2[2]};
  apply(c, M, v, w, 0.0, dtw, zero);
  /* rolling */
  side_velocities(c, v, w, va, wa, vb, wb);
  double yr[3];
  for (int i = 0; i < 3; ++i) yr[i] = c->lr[i] - ((wb[i] - wa[i]) + c->sr * c->lr[i]) / c->Dr;
  project_ball(yr, 3, c->rmu * fabs(c->ln));
  double dr[3] = {yr[0] - c->lr[0], yr[1] - c->lr[1], yr[2] - c->lr[2]};
  for (int i = 0; i < 3; ++i) c->lr[i] = yr[i];
  apply(c, M, v, w, 0.0, zero, dr);
}

/* Diagonally scaled natural-map residual (a Jacobi pass; order-free):
 * |Lambda - Pi_B(Lambda - D^-1 w(Lambda))| / max(|Lambda|, 1e-12).
 * Per contact: e = its squared natural-map entries, l = its squared impulses. */
static void residual_terms(const contact *c, const double *v, const double *w, double *e_out,
                           double *l_out) {
  {
    double va[3], wa[3], vb[3], wb[3];
    side_velocities(c, v, w, va, wa, vb, wb);
    double dv[3] = {vb[0] - va[0], vb[1] - va[1], vb[2] - va[2]};
    double wn = dot3(c->n, dv) + c->Sn * c->ln - c->qn;
    double pn = c->ln - wn / c->Dn;
    if (pn < -c->fc) pn = -c->fc;
    double u[3];
    slip_velocity(c, va, wa, vb, wb, u);
    double yt[2] = {c->lt[0] - (dot3(c->t1, u) + c->st * c->lt[0]) / c->Dt,
                    c->lt[1] - (dot3(c->t2, u) + c->st * c->lt[1]) / c->Dt};
    project_ball(yt, 2, c->mu * fabs(c->ln));
    double yr[3];
    for (int i = 0; i < 3; ++i) yr[i] = c->lr[i] - ((wb[i] - wa[i]) + c->sr * c->lr[i]) / c->Dr;
    project_ball(yr, 3, c->rmu * fabs(c->ln));
    double e = (c->ln - pn) * (c->ln - pn);
    for (int i = 0; i < 2; ++i) e += (c->lt[i] - yt[i]) * (c->lt[i] - yt[i]);
    for (int i = 0; i < 3; ++i) e += (c->lr[i] - yr[i]) * (c->lr[i] - yr[i]);
    *e_out = e;
    *l_out = c->ln * c->ln + c->lt[0] * c->lt[0] + c->lt[1] * c->lt[1] +
             c->lr[0] * c->lr[0] + c->lr[1] * c->lr[1] + c->lr[2] * c->lr[2];
  }
}

/* The sums run over the contacts in key order; with threads > 1 the terms
 * are computed in parallel (scratch holds 2 nc doubles) and then summed in
 * that same order, so the value does not depend on the thread count. */
static double residual(const contact *C, int nc, const double *v, const double *w, int threads,
                       double *scratch) {
  double num = 0.0, den = 0.0;
  if (threads > 1 && scratch) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads) schedule(static)
#endif
    for (int k = 0; k < nc; ++k) residual_terms(&C[k], v, w, &scratch[2 * k], &scratch[2 * k + 1]);
    for (int k = 0; k < nc; ++k) { num += scratch[2 * k]; den += scratch[2 * k + 1]; }
  } else {
    for (int k = 0; k < nc; ++k) {
      double e, l;
      residual_terms(&C[k], v, w, &e, &l);
      num += e;
      den += l;
    }
  }
  double d = sqrt(den);
  return sqrt(num) / (d > 1e-12 ? d : 1e-12);
}

/* ------------------------------------------------------------------ */
/* Colouring: colour(c) = smallest colour not used by a neighbour of    */
/* higher priority (neighbours share a dynamic particle). Computed by   */
/* plain sequential greedy colouring in decreasing priority order.      */
/* Incremental steps keep the colour of every contact whose key existed */
/* in the previous step (two such contacts share a particle now iff     */
/* they did then, so the kept colours stay a proper colouring) and      */
/* colour only the new contacts, greedily in decreasing priority: the   */
/* smallest colour used by no neighbour that is kept or new and of      */
/* higher priority.                                                     */
/* ------------------------------------------------------------------ */
static contact *g_sort_base;
static int cmp_prio_desc(const void *pa, const void *pb) {
  const contact *a = &g_sort_base[*(const int *)pa], *b = &g_sort_base[*(const int *)pb];
  if (a->prio != b->prio) return a->prio > b->prio ? -1 : 1;
  return a->key > b->key ? -1 : (a->key < b->key ? 1 : 0);
}

static int colour_contacts(contact *C, int nc, int n) {
  int *deg = (int *)calloc(n + 1, sizeof(int));
  int *start = (int *)calloc(n + 1, sizeof(int));
  int *fill = (int *)calloc(n + 1, sizeof(int));
  int *inc = (int *)malloc(sizeof(int) * (2 * nc + 1));
  int *ord = (int *)malloc(sizeof(int) * (nc + 1));
  int ncol = 0;
  if (!deg || !start || !fill || !inc || !ord) { ncol = -1; goto out; }
  for (int k = 0; k < nc; ++k) {
    deg[C[k].a]++;
    if (C[k].b >= 0) deg[C[k].b]++;
  }
  for (int i = 0; i < n; ++i) start[i + 1] = start[i] + deg[i];
  for (int k = 0; k < nc; ++k) {
    inc[start[C[k].a] + fill[C[k].a]++] = k;
    if (C[k].b >= 0) inc[start[C[k].b] + fill[C[k].b]++] = k;
  }
  for (int k = 0; k < nc; ++k) { ord[k] = k; C[k].colour = C[k].kept_colour; }
  g_sort_base = C;
  qsort(ord, nc, sizeof(int), cmp_prio_desc);
  {
    int cap = 64;
    unsigned char *used = (unsigned char *)calloc(cap, 1);
    if (!used) { ncol = -1; goto out; }
    for (int o = 0; o < nc; ++o) {
      contact *c = &C[ord[o]];
      if (c->colour >= 0) {  /* kept from the previous step */
        if (c->colour + 1 > ncol) ncol = c->colour + 1;
        continue;
      }
      int ends[2] = {c->a, c->b};
      for (int e = 0; e < 2; ++e) {
        if (ends[e] < 0) continue;
        for (int m = start[ends[e]]; m < start[ends[e] + 1]; ++m) {
          int col = C[inc[m]].colour;
          if (col < 0) continue; /* not yet coloured: a new contact of lower priority */
          if (col >= cap) {
            int ncap = 2 * col + 2;
            unsigned char *nu = (unsigned char *)realloc(used, ncap);
            if (!nu) { free(used); ncol = -1; goto out; }
            memset(nu + cap, 0, ncap - cap);
            used = nu; cap = ncap;
          }
          used[col] = 1;
        }
      }
      int col = 0;
      while (col < cap && used[col]) ++col;
      c->colour = col;
      if (col + 1 > ncol) ncol = col + 1;
      /* clear the marks */
      for (int e = 0; e < 2; ++e) {
        if (ends[e] < 0) continue;
        for (int m = start[ends[e]]; m < start[ends[e] + 1]; ++m) {
          int cc = C[inc[m]].colour;
          if (cc >= 0 && cc < cap) used[cc] = 0;
        }
      }
    }
    free(used);
  }
out:
  free(deg); free(start); free(fill); free(inc); free(ord);
  return ncol;
}

/* ------------------------------------------------------------------ */
/* The step                                                             */
/* ------------------------------------------------------------------ */
static int find_key(int n, const uint64_t *keys, uint64_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = lo + (hi - lo) / 2;
    if (keys[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < n && keys[lo] == key) ? lo : -1;
}

static uint64_t lcg_next(uint64_t *s) {
  *s = *s * 6364136223846793005ull + 1442695040888963407ull;
  return *s >> 33;
}

/* ------------------------------------------------------------------ */
/* Learned warm start: per-contact features and the impulse scale      */
/* ------------------------------------------------------------------ */
/* Surface columns: the heightfield cells grouped f x f, f the smallest
 * integer with f * cell >= 4 r_max; the surface of a column is the largest
 * z + r of its particles (FP32, exact max). */
static int column_of(const orc_params *P, int f, float px, float py, int ncx, int ncy) {
  float w = P->hf_cell * (float)f;
  float tx = (px - P->hf_x0) / w, ty = (py - P->hf_y0) / w;
  float fx = floorf(tx), fy = floorf(ty);
  int i, j;
  if (!(fx >= 0.0f)) i = 0; else if (fx > (float)(ncx - 1)) i = ncx - 1; else i = (int)fx;
  if (!(fy >= 0.0f)) j = 0; else if (fy > (float)(ncy - 1)) j = ncy - 1; else j = (int)fy;
  return j * ncx + i;
}

int32_t orc_column_factor(const orc_params *P, int32_t n, const double *r) {
  double rmax = 0.0;
  for (int i = 0; i < n; ++i) if ((double)(float)r[i] > rmax) rmax = (double)(float)r[i];
  if (P->hf_nx <= 0 || !(P->hf_cell > 0.0f)) return 0;
  int f = (int)ceil(4.0 * rmax / (double)P->hf_cell);
  return f < 1 ? 1 : f;
}

/* Features (one row per contact, section "learned warm start" of the
 * design): (J_n v^*) / (|g| h), delta/dbar, Lambda_n0/W, |Lambda_t0|/W,
 * (Lambda_t0 . s)/W, persisted, Z_a, Z_b, depth below surface/dbar, type;
 * W = m_eff |g| h with m_eff = 1/(1/m_a + 1/m_b); s = unit tangential slip
 * velocity at v^* (or, below 1e-6 m/s, the unit n x e_k with e_k the axis
 * least aligned with n). v and w hold v^* and w_n. */
static int contact_features(const orc_params *P, int n, const double *x, const double *r,
                            const masses *M, const double *v, const double *w, contact *C,
                            int nc) {
  double gn = sqrt(dot3(P->gravity, P->gravity));
  double h = P->dt;
  int *Z = (int *)calloc(n + 1, sizeof(int));
  if (!Z) return -1;
  for (int k = 0; k < nc; ++k) { Z[C[k].a]++; if (C[k].b >= 0) Z[C[k].b]++; }
  int f = orc_column_factor(P, n, r), ncx = 0, ncy = 0;
  float *surf = NULL;
  if (f > 0) {
    ncx = (P->hf_nx + f - 1) / f;
    ncy = (P->hf_ny + f - 1) / f;
    surf = (float *)malloc(sizeof(float) * ncx * ncy);
    if (!surf) { free(Z); return -1; }
    for (int q = 0; q < ncx * ncy; ++q) surf[q] = -INFINITY;
    for (int i = 0; i < n; ++i) {
      if (!(r[i] > 0.0)) continue;  /* dormant */
      int col = column_of(P, f, (float)x[3 * i], (float)x[3 * i + 1], ncx, ncy);
      float top = (float)x[3 * i + 2] + (float)r[i];
      if (top > surf[col]) surf[col] = top;
    }
  }
  for (int k = 0; k < nc; ++k) {
    contact *c = &C[k];
    double va[3], wa[3], vb[3], wb[3], u[3];
    side_velocities(c, v, w, va, wa, vb, wb);
    double dv[3] = {vb[0] - va[0], vb[1] - va[1], vb[2] - va[2]};
    slip_velocity(c, va, wa, vb, wb, u);
    double un = dot3(u, c->n);
    double ut[3] = {u[0] - un * c->n[0], u[1] - un * c->n[1], u[2] - un * c->n[2]};
    double ms = norm3(ut);
    if (ms > 1e-6) {
      for (int i = 0; i < 3; ++i) c->sdir[i] = ut[i] / ms;
    } else {
      int ax = 0;
      double best = fabs(c->n[0]);
      if (fabs(c->n[1]) < best) { best = fabs(c->n[1]); ax = 1; }
      if (fabs(c->n[2]) < best) ax = 2;
      double e[3] = {0.0, 0.0, 0.0}, t[3];
      e[ax] = 1.0;
      cross3(c->n, e, t);
      double s = norm3(t);
      for (int i = 0; i < 3; ++i) c->sdir[i] = t[i] / s;
    }
    double imb = c->b >= 0 ? M->m_inv[c->b] : 0.0;
    c->W = gn * h / (M->m_inv[c->a] + imb);
    double ra = r[c->a], dbar = c->b >= 0 ? ra + r[c->b] : 2.0 * ra;
    double lt[3];
    for (int i = 0; i < 3; ++i) lt[i] = c->lt[0] * c->t1[i] + c->lt[1] * c->t2[i];
    double depth = 0.0;
    if (surf) {
      int col = column_of(P, f, (float)x[3 * c->a], (float)x[3 * c->a + 1], ncx, ncy);
      depth = ((double)surf[col] - x[3 * c->a + 2]) / dbar;
    }
    c->feat[0] = dot3(c->n, dv) / (gn * h);
    c->feat[1] = c->delta / dbar;
    c->feat[2] = c->ln / c->W;
    c->feat[3] = norm3(lt) / c->W;
    c->feat[4] = dot3(lt, c->sdir) / c->W;
    c->feat[5] = c->persisted ? 1.0 : 0.0;
    c->feat[6] = (double)Z[c->a];
    c->feat[7] = c->b >= 0 ? (double)Z[c->b] : 0.0;
    c->feat[8] = depth;
    c->feat[9] = c->b >= 0 ? 0.0 : (c->is_tool ? 2.0 : 1.0);
  }
  free(surf);
  free(Z);
  return 0;
}

/* Impact stage (the Newton impact law, section "Contacting rigid
 * multibodies"), a velocity-level solve before the main one. A contact whose
 * approach speed at the start of the step, -G_n v_n, exceeds v_imp is an
 * impact and gets the target G_n v+ = e (-G_n v_n); every other normal row is
 * held at G_n v+ >= 0; friction and rolling keep their cones; no cohesion.
 * Rigid rows (no compliance), impulses from zero, impact_iters sweeps in the
 * main solve's order, acting on the predicted velocities v*. Afterwards the
 * main solve's q_n = -(4/h) Upsilon g + Upsilon G_n v takes the post-impact
 * velocities: q_n += Upsilon (G_n v+ - G_n v*). Returns the number of
 * impacts (0: nothing done). */
static int impact_stage(const orc_params *P, contact *C, int nc, const int *order, const masses *M,
                        double *v, double *w) {
  int nimp = 0;
  for (int k = 0; k < nc; ++k) nimp += -C[k].Gvn > P->impact_speed;
  if (P->impact_iters <= 0 || nimp == 0) return 0;
  contact *I = (contact *)malloc(sizeof(contact) * (nc + 1));
  double *gv = (double *)malloc(sizeof(double) * (nc + 1));
  if (!I || !gv) { free(I); free(gv); return -1; }
  double va[3], wa[3], vb[3], wb[3];
  for (int k = 0; k < nc; ++k) {
    I[k] = C[k];
    contact *c = &I[k];
    side_velocities(c, v, w, va, wa, vb, wb);
    double dv[3] = {vb[0] - va[0], vb[1] - va[1], vb[2] - va[2]};
    gv[k] = dot3(c->n, dv);
    c->Dn -= c->Sn;   /* rigid normal row */
    c->Sn = 0.0;
    c->qn = -c->Gvn > P->impact_speed ? P->restitution * (-c->Gvn) : 0.0;
    c->fc = 0.0;      /* no cohesion */
    c->ln = 0.0; c->lt[0] = c->lt[1] = 0.0; c->lr[0] = c->lr[1] = c->lr[2] = 0.0;
  }
  for (int it = 0; it < P->impact_iters; ++it)
    for (int k = 0; k < nc; ++k) pgs_contact(&I[order[k]], M, v, w);
  double tau = 2.0 * P->dt, ups = 1.0 / (1.0 + 4.0 * tau / P->dt);
  for (int k = 0; k < nc; ++k) {
    contact *c = &C[k];
    side_velocities(c, v, w, va, wa, vb, wb);
    double dv[3] = {vb[0] - va[0], vb[1] - va[1], vb[2] - va[2]};
    c->qn += ups * (dot3(c->n, dv) - gv[k]);
  }
  free(I); free(gv);
  return nimp;
}

int32_t orc_step(const orc_params *P, int32_t n, double *x, double *v, double *w,
                 const double *r, int32_t n_prev, const uint64_t *prev_keys,
                 const double *prev_lam, const int32_t *prev_colour, int32_t step_index,
                 int32_t cap, uint64_t *out_keys,
                 double *out_lam, int32_t *out_colour, double *out_delta,
                 double *out_feat, double *out_targ, orc_stats *st) {
  if (!P || n < 0 || cap < 0 || !st || (n > 0 && (!x || !v || !w || !r))) return -2;
  if (n_prev > 0 && (!prev_keys || !prev_lam)) return -2;
  /* incremental colouring: every step but each recolour_every-th (counting
   * from the first, step_index 0) keeps the previous step's colours */
  const int incremental = P->recolour_every > 1 && step_index > 0 && step_index % P->recolour_every != 0;
  if (incremental && n_prev > 0 && !prev_colour) return -2;
  memset(st, 0, sizeof(*st));
  int rc = 0, nb = 0;
  double h = P->dt;
  wbox *B = world_boxes(P, &nb);
  masses M = {NULL, NULL};
  uint64_t *keys = NULL;
  contact *C = NULL;
  int *order = NULL, *cstart = NULL;
  if (!B) return -2;
  M.m_inv = (double *)malloc(sizeof(double) * (n + 1));
  M.I_inv = (double *)malloc(sizeof(double) * (n + 1));
  keys = (uint64_t *)malloc(sizeof(uint64_t) * (cap + 1));
  if (!M.m_inv || !M.I_inv || !keys) { rc = -2; goto done; }
  for (int i = 0; i < n; ++i) {
    if (!(r[i] > 0.0)) { M.m_inv[i] = M.I_inv[i] = 0.0; continue; }  /* dormant */
    double m = P->density * 4.0 / 3.0 * ORC_PI * r[i] * r[i] * r[i];
    M.m_inv[i] = 1.0 / m;
    M.I_inv[i] = 1.0 / (0.4 * m * r[i] * r[i]);
  }
  /* 1. collision detection on x_n */
  keylist L = {keys, 0, cap, 0};
  rc = detect(P, n, x, r, 0, B, nb, &L);
  if (rc) goto done;
  if (L.overflow) { rc = -1; goto done; }
  int nc = L.n;
  qsort(keys, nc, sizeof(uint64_t), cmp_u64);
  C = (contact *)calloc(nc + 1, sizeof(contact));
  if (!C) { rc = -2; goto done; }
  double *v0 = (double *)malloc(sizeof(double) * 3 * (n + 1));
  if (!v0) { rc = -2; goto done; }
  memcpy(v0, v, sizeof(double) * 3 * n);
  for (int k = 0; k < nc; ++k) {
    contact *c = &C[k];
    c->key = keys[k];
    c->prio = orc_priority(keys[k]);
    c->a = (int)(keys[k] >> 32);
    uint32_t lo = (uint32_t)(keys[k] & 0xFFFFFFFFu);
    if (lo & ORC_STATIC_BIT) {
      c->b = -1;
      c->surf = (int)(lo & ~ORC_STATIC_BIT);
      c->is_tool = c->surf >= 1 + P->n_walls;
      st->n_static++;
    } else {
      c->b = (int)lo;
      c->surf = -1;
      c->is_tool = 0;
      st->n_pp++;
    }
    contact_geometry(P, B, x, r, c);
    contact_rows(P, r, &M, v0, c);
    c->kept_colour = -1;
    if (incremental && n_prev > 0) {
      int j = find_key(n_prev, prev_keys, c->key);
      if (j >= 0) c->kept_colour = prev_colour[j];
    }
  }
  free(v0);
  /* 2. p = M v_n + h f: v^* = v_n + h g (gravity is the only external force) */
  for (int i = 0; i < n; ++i)
    if (r[i] > 0.0)
      for (int k = 0; k < 3; ++k) v[3 * i + k] += h * P->gravity[k];
  /* 3. warm start: previous impulses by key, Lambda_t re-projected onto the
   *    new tangent plane, all clamped into the new bounds (v += M^-1 G^T
   *    lambda_0 follows the impact stage below) */
  for (int k = 0; k < nc; ++k) {
    contact *c = &C[k];
    c->ln = 0.0; c->lt[0] = c->lt[1] = 0.0; c->lr[0] = c->lr[1] = c->lr[2] = 0.0;
    if (!P->warm_start || n_prev <= 0) continue;
    int j = find_key(n_prev, prev_keys, c->key);
    if (j < 0) continue;
    const double *pl = prev_lam + 7 * j;
    c->persisted = 1;
    c->ln = pl[0] < -c->fc ? -c->fc : pl[0];
    double tw[3] = {pl[1], pl[2], pl[3]};
    c->lt[0] = dot3(c->t1, tw);
    c->lt[1] = dot3(c->t2, tw);
    project_ball(c->lt, 2, c->mu * fabs(c->ln));
    for (int i = 0; i < 3; ++i) c->lr[i] = pl[4 + i];
    project_ball(c->lr, 3, c->rmu * fabs(c->ln));
  }
  /* learned-warm-start features of every contact at v* with lambda_0 */
  if (contact_features(P, n, x, r, &M, v, w, C, nc)) { rc = -2; goto done; }
  /* 4. colouring and the sweep order */
  int ncol = colour_contacts(C, nc, n);
  if (ncol < 0) { rc = -2; goto done; }
  st->n_colours = ncol;
  order = (int *)malloc(sizeof(int) * (nc + 1));
  cstart = (int *)calloc(ncol + 2, sizeof(int));
  if (!order || !cstart) { rc = -2; goto done; }
  if (P->order == 1) {
    for (int k = 0; k < nc; ++k) order[k] = k; /* ascending key */
  } else {
    for (int k = 0; k < nc; ++k) cstart[C[k].colour + 1]++;
    for (int c = 0; c < ncol; ++c) cstart[c + 1] += cstart[c];
    int *fill = (int *)calloc(ncol + 1, sizeof(int));
    if (!fill) { rc = -2; goto done; }
    for (int k = 0; k < nc; ++k) order[cstart[C[k].colour] + fill[C[k].colour]++] = k;
    free(fill);
    if (P->shuffle_seed) {
      uint64_t s = P->shuffle_seed;
      for (int c = 0; c < ncol; ++c) {
        int lo = cstart[c], cnt = cstart[c + 1] - cstart[c];
        for (int i = cnt - 1; i > 0; --i) {
          int j = (int)(lcg_next(&s) % (uint64_t)(i + 1));
          int t = order[lo + i]; order[lo + i] = order[lo + j]; order[lo + j] = t;
        }
      }
    }
  }
  /* impact stage on v*, then the warm start v += M^-1 G^T lambda_0 */
  st->impacts = impact_stage(P, C, nc, order, &M, v, w);
  if (st->impacts < 0) { rc = -2; goto done; }
  for (int k = 0; k < nc; ++k) {
    contact *c = &C[k];
    if (!c->persisted) continue;
    double tw0[3] = {c->lt[0] * c->t1[0] + c->lt[1] * c->t2[0],
                     c->lt[0] * c->t1[1] + c->lt[1] * c->t2[1],
                     c->lt[0] * c->t1[2] + c->lt[1] * c->t2[2]};
    apply(c, &M, v, w, c->ln, tw0, c->lr);
  }
  /* 5. PGS sweeps. With threads > 1 (a timing option of the CPU baseline,
   *    colour order only) the contacts of one colour are updated by several
   *    threads: they share no particle, so the result is the serial one bit
   *    for bit. */
  int it = 0;
  double res = -1.0;
  int every = P->residual_every > 0 ? P->residual_every : 1;
  int threads = (P->threads > 1 && P->order == 0) ? P->threads : 1;
  double *rs = threads > 1 ? (double *)malloc(sizeof(double) * 2 * (nc + 1)) : NULL;
  if (threads > 1 && !rs) { rc = -2; goto done; }
  while (it < P->iters) {
    if (threads > 1) {
      for (int col = 0; col < ncol; ++col) {
        const int lo = cstart[col], hi = cstart[col + 1];
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads) schedule(static)
#endif
        for (int k = lo; k < hi; ++k) pgs_contact(&C[order[k]], &M, v, w);
      }
    } else {
      for (int k = 0; k < nc; ++k) pgs_contact(&C[order[k]], &M, v, w);
    }
    ++it;
    if (P->tol > 0.0 && it % every == 0) {
      res = residual(C, nc, v, w, threads, rs);
      if (res <= P->tol) break;
    }
  }
  st->iterations = it;
  st->residual = residual(C, nc, v, w, threads, rs);
  free(rs);
  /* 6. tool force and torque (soil on tool) */
  for (int k = 0; k < nc; ++k) {
    const contact *c = &C[k];
    if (!c->is_tool) continue;
    double Fi[3], arm[3], tq[3];
    for (int i = 0; i < 3; ++i)
      Fi[i] = (c->ln * c->n[i] + c->lt[0] * c->t1[i] + c->lt[1] * c->t2[i]) / h;
    for (int i = 0; i < 3; ++i) arm[i] = c->xc[i] - P->tool_pos[i];
    cross3(arm, Fi, tq);
    for (int i = 0; i < 3; ++i) {
      st->tool_force[i] += Fi[i];
      st->tool_torque[i] += tq[i] + c->lr[i] / h;
    }
  }
  /* 7. x_{n+1} = x_n + h v_{n+1} */
  for (int i = 0; i < n; ++i)
    if (r[i] > 0.0)
      for (int k = 0; k < 3; ++k) x[3 * i + k] += h * v[3 * i + k];
  /* outputs in ascending key order */
  st->n_contacts = nc;
  for (int k = 0; k < nc; ++k) {
    const contact *c = &C[k];
    if (out_keys) out_keys[k] = c->key;
    if (out_lam) {
      double *o = out_lam + 7 * k;
      o[0] = c->ln;
      for (int i = 0; i < 3; ++i) o[1 + i] = c->lt[0] * c->t1[i] + c->lt[1] * c->t2[i];
      for (int i = 0; i < 3; ++i) o[4 + i] = c->lr[i];
    }
    if (out_colour) out_colour[k] = c->colour;
    if (out_delta) out_delta[k] = c->delta;
    if (out_feat)
      for (int i = 0; i < 10; ++i) out_feat[10 * k + i] = c->feat[i];
    if (out_targ) {
      double lt[3], nxs[3];
      for (int i = 0; i < 3; ++i) lt[i] = c->lt[0] * c->t1[i] + c->lt[1] * c->t2[i];
      cross3(c->n, c->sdir, nxs);
      out_targ[3 * k + 0] = c->ln / c->W;
      out_targ[3 * k + 1] = dot3(lt, c->sdir) / c->W;
      out_targ[3 * k + 2] = dot3(lt, nxs) / c->W;
    }
  }
done:
  free(B); free(M.m_inv); free(M.I_inv); free(keys); free(C); free(order); free(cstart);
  return rc;
}

/* ------------------------------------------------------------------ */
/* MLP 10 -> 64 -> 64 -> 3 with ReLU, FP64 forward and backward          */
/* ------------------------------------------------------------------ */
#define MLP_IN 10
#define MLP_H 64
#define MLP_OUT 3

static void mlp_layers(const double *x, const double *W1, const double *b1,
                       const double *W2, const double *b2, const double *W3,
                       const double *b3, double z1[MLP_H], double a1[MLP_H],
                       double z2[MLP_H], double a2[MLP_H], double y[MLP_OUT]) {
  for (int o = 0; o < MLP_H; ++o) {
    double s = b1[o];
    for (int i = 0; i < MLP_IN; ++i) s += W1[o * MLP_IN + i] * x[i];
    z1[o] = s;
    a1[o] = s > 0.0 ? s : 0.0;
  }
  for (int o = 0; o < MLP_H; ++o) {
    double s = b2[o];
    for (int i = 0; i < MLP_H; ++i) s += W2[o * MLP_H + i] * a1[i];
    z2[o] = s;
    a2[o] = s > 0.0 ? s : 0.0;
  }
  for (int o = 0; o < MLP_OUT; ++o) {
    double s = b3[o];
    for (int i = 0; i < MLP_H; ++i) s += W3[o * MLP_H + i] * a2[i];
    y[o] = s;
  }
}

void orc_mlp_forward(int32_t m, const double *X, const double *W1, const double *b1,
                     const double *W2, const double *b2, const double *W3,
                     const double *b3, double *Y) {
  double z1[MLP_H], a1[MLP_H], z2[MLP_H], a2[MLP_H];
  for (int s = 0; s < m; ++s)
    mlp_layers(X + MLP_IN * s, W1, b1, W2, b2, W3, b3, z1, a1, z2, a2, Y + MLP_OUT * s);
}

double orc_mlp_loss_grad(int32_t m, const double *X, const double *T,
                         const double *W1, const double *b1, const double *W2,
                         const double *b2, const double *W3, const double *b3,
                         double *gW1, double *gb1, double *gW2, double *gb2,
                         double *gW3, double *gb3) {
  memset(gW1, 0, sizeof(double) * MLP_H * MLP_IN);
  memset(gb1, 0, sizeof(double) * MLP_H);
  memset(gW2, 0, sizeof(double) * MLP_H * MLP_H);
  memset(gb2, 0, sizeof(double) * MLP_H);
  memset(gW3, 0, sizeof(double) * MLP_OUT * MLP_H);
  memset(gb3, 0, sizeof(double) * MLP_OUT);
  double loss = 0.0;
  double scale = 1.0 / (3.0 * (double)(m > 0 ? m : 1));
  for (int s = 0; s < m; ++s) {
    const double *x = X + MLP_IN * s;
    double z1[MLP_H], a1[MLP_H], z2[MLP_H], a2[MLP_H], y[MLP_OUT];
    mlp_layers(x, W1, b1, W2, b2, W3, b3, z1, a1, z2, a2, y);
    double dy[MLP_OUT];
    for (int o = 0; o < MLP_OUT; ++o) {
      double e = y[o] - T[MLP_OUT * s + o];
      loss += e * e * scale;
      dy[o] = 2.0 * e * scale;
    }
    double da2[MLP_H];
    for (int i = 0; i < MLP_H; ++i) da2[i] = 0.0;
    for (int o = 0; o < MLP_OUT; ++o) {
      gb3[o] += dy[o];
      for (int i = 0; i < MLP_H; ++i) {
        gW3[o * MLP_H + i] += dy[o] * a2[i];
        da2[i] += W3[o * MLP_H + i] * dy[o];
      }
    }
    double dz2[MLP_H], da1[MLP_H];
    for (int i = 0; i < MLP_H; ++i) { dz2[i] = z2[i] > 0.0 ? da2[i] : 0.0; da1[i] = 0.0; }
    for (int o = 0; o < MLP_H; ++o) {
      gb2[o] += dz2[o];
      for (int i = 0; i < MLP_H; ++i) {
        gW2[o * MLP_H + i] += dz2[o] * a1[i];
        da1[i] += W2[o * MLP_H + i] * dz2[o];
      }
    }
    for (int o = 0; o < MLP_H; ++o) {
      double dz1 = z1[o] > 0.0 ? da1[o] : 0.0;
      gb1[o] += dz1;
      for (int i = 0; i < MLP_IN; ++i) gW1[o * MLP_IN + i] += dz1 * x[i];
    }
  }
  return loss;
}
