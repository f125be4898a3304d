/*
 * tds_oracle.h -- the CPU oracle for one time step of the active-soil
 * particle system of "A multiscale model of terrain dynamics for real-time
 * earthmoving simulation" (Servin, Berglund, Nystedt).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow FP64 restatement of the
 * method (single-threaded unless asked to update the contacts of a colour on
 * several threads, which gives the same bits), written to judge the CUDA path. Only the test
 * suite, the package smoke check and the benchmark's CPU-baseline leg may
 * load it. It shares no code, header, table or helper with the CUDA library.
 *
 * What one step computes (the collision detection, PGS solve of the
 * mesoscale MCP and position update of the particle step, Algorithm 1):
 *   1. contact detection (particle-particle, particle-heightfield,
 *      particle-box) with an FP32 predicate that the CUDA path evaluates
 *      bit-identically;
 *   2. per-contact rows of the nonsmooth DEM contact law (Eqs. signCoul1-3)
 *      with the Hertz mapping of the normal row and the SPOOK coefficients
 *      (section "Contacting rigid multibodies");
 *   3. greedy colouring of the contact graph in decreasing hashed priority;
 *   4. projected Gauss-Seidel sweeps, colour by colour (or in plain key
 *      order for the sequential reference);
 *   5. x_{n+1} = x_n + dt v_{n+1}.
 *
 * Readings where the paper is silent or garbled are listed next to the code
 * that takes them.
 */
#ifndef TDS_ORACLE_H
#define TDS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Everything a step needs besides the particle state. FP32 fields are the
 * geometry that the FP32 contact predicate reads; FP64 fields are physics. */
typedef struct {
  double density, young, poisson;     /* rho [kg/m^3], E [Pa], nu */
  double mu_t, mu_r, cohesion;        /* friction, rolling resistance, c_p [Pa] */
  double mu_tool;                     /* friction against the tool */
  double dt;                          /* h [s] */
  double gravity[3];                  /* [m/s^2] */
  double gamma_t, gamma_r;            /* velocity-row regularisation (paper silent) */
  int32_t iters;                      /* sweeps (fixed mode) or cap (residual mode) */
  int32_t residual_every;             /* residual check period in residual mode */
  double tol;                         /* <= 0: fixed sweeps; > 0: stop at residual <= tol */
  int32_t order;                      /* 0: colour sweep, 1: sequential key order */
  int32_t warm_start;                 /* 0: cold, 1: previous-step impulses by key */
  uint64_t shuffle_seed;              /* != 0: permute contacts inside each colour */
  /* heightfield: (nx+1)*(ny+1) FP32 heights, h[j*(nx+1)+i]; nx == 0 disables it */
  int32_t hf_nx, hf_ny;
  float hf_x0, hf_y0, hf_cell;
  const float *hf_h;
  /* static walls: world frame, 10 floats each: center[3], quat[4] (w,x,y,z), half[3] */
  int32_t n_walls;
  const float *walls;
  /* kinematic tool: boxes in the tool frame (10 floats each) and its motion */
  int32_t n_tool;
  const float *tool_boxes;
  float tool_pos[3], tool_quat[4], tool_vel[3], tool_angvel[3];
  /* impact stage (section "Contacting rigid multibodies", Newton impact law):
   * impact_iters == 0 disables it */
  double restitution;                 /* e */
  double impact_speed;                /* v_imp [m/s] */
  int32_t impact_iters;               /* sweeps of the impact solve */
  /* threads updating the contacts of one colour at a time (<= 1: one; a
   * timing option, the results are the same bit for bit; colour order only) */
  int32_t threads;
  /* colouring: every recolour_every-th step (and the first) colours every
   * contact; the steps between keep the previous step's colour of each
   * contact whose key existed then and colour only the new ones (<= 1: every
   * step colours every contact) */
  int32_t recolour_every;
} orc_params;

typedef struct {
  int32_t n_contacts, n_pp, n_static, n_colours, iterations;
  double residual;
  double tool_force[3], tool_torque[3];
  int32_t impacts;                    /* contacts treated as impacts this step */
} orc_stats;

/* Contact keys: ((uint64)a << 32) | b for particles a < b, and
 * ((uint64)a << 32) | 0x80000000 | s for particle a against static surface s
 * (s = 0 heightfield, 1..n_walls walls, then the tool boxes). */
#define ORC_STATIC_BIT 0x80000000u

/* Contact detection only. x: n*3 positions, r: n radii (FP64 copies of FP32
 * values; the predicate rounds them to float). brute != 0 tests every pair.
 * Writes up to cap keys in ascending order; returns the count, or -1 if cap
 * is too small, -2 on bad arguments or allocation failure. */
int32_t orc_find_contacts(const orc_params *P, int32_t n, const double *x,
                          const double *r, int32_t brute, int32_t cap,
                          uint64_t *keys);

/* One time step, in place on x, v, w (n*3 each, FP64); r: radii.
 * prev_keys (ascending) / prev_lam (7 per key: Lambda_n, Lambda_t world xyz,
 * Lambda_r xyz) / prev_colour give the previous step's impulses for the warm
 * start and its colours for incremental colouring; step_index counts the
 * steps taken before this one.
 * Outputs, in ascending key order, up to cap contacts: keys, lam (7 each),
 * colour, delta (overlap). Returns 0, -1 if cap is too small, -2 on bad
 * arguments or allocation failure. */
int32_t orc_step(const orc_params *P, int32_t n, double *x, double *v, double *w,
                 const double *r, int32_t n_prev, const uint64_t *prev_keys,
                 const double *prev_lam, const int32_t *prev_colour, int32_t step_index,
                 int32_t cap, uint64_t *out_keys,
                 double *out_lam, int32_t *out_colour, double *out_delta,
                 double *out_feat, double *out_targ, orc_stats *st);

/* Learned warm start. out_feat (10 per contact) and out_targ (3 per contact)
 * of orc_step, in key order:
 *   features: (J_n v^*) / (|g| h), delta/dbar, Lambda_n0/W, |Lambda_t0|/W,
 *             (Lambda_t0 . s)/W, persisted (0/1), Z_a, Z_b (0 static),
 *             depth below the surface / dbar, type (0 pair, 1 terrain or wall,
 *             2 tool);
 *   targets:  Lambda_n/W, (Lambda_t . s)/W, (Lambda_t . (n x s))/W of the
 *             step's final impulses;
 * with W = |g| h / (1/m_a + 1/m_b), dbar = r_a + r_b (static 2 r_a), lambda_0
 * the previous-step impulses as the warm start sets them, v^* = v_n + h g, s
 * the unit tangential slip velocity at v^* (below 1e-6 m/s: unit n x e_k, e_k
 * the axis least aligned with n). Surface columns are the heightfield cells
 * grouped f x f (orc_column_factor), the surface of a column the largest
 * FP32 z + r of its particles. */
int32_t orc_column_factor(const orc_params *P, int32_t n, const double *r);

/* The SplitMix64 finaliser used as the colouring priority of a key. */
uint64_t orc_priority(uint64_t key);

/* ---- learned warm start: the 10 -> 64 -> 64 -> 3 ReLU MLP ----------------
 * Row-major weights: W1[64][10], b1[64], W2[64][64], b2[64], W3[3][64], b3[3].
 * Forward on m rows of 10 features; y: m*3. */
void orc_mlp_forward(int32_t m, const double *X, const double *W1, const double *b1,
                     const double *W2, const double *b2, const double *W3,
                     const double *b3, double *Y);
/* Mean-squared-error loss L = (1/(3m)) sum (y - t)^2 and its gradients with
 * respect to every weight and bias (same shapes as the weights). */
double orc_mlp_loss_grad(int32_t m, const double *X, const double *T,
                         const double *W1, const double *b1, const double *W2,
                         const double *b2, const double *W3, const double *b3,
                         double *gW1, double *gb1, double *gW2, double *gb2,
                         double *gW3, double *gb3);

#ifdef __cplusplus
}
#endif
#endif
