/*
 * tds.h -- C ABI of libtds, the GB300 (sm_103a) time step of the active-soil
 * particle system from "A multiscale model of terrain dynamics for real-time
 * earthmoving simulation" (Servin, Berglund, Nystedt).
 *
 * The mesoscale model of the paper takes the equipment's motion and contact
 * interfaces as input (section "Mesoscale model": the macroscale model
 * supplies the equipment's motion and contact forces at the terrain
 * interface) together with the terrain surface heightfield (Eq. surface),
 * and returns the soil motion (particles) and the body-particle contact force
 * that is the source of the digging resistance (section "Microscale model").
 * One call of tds_step performs, per time step, the three parts of the
 * particle step in Algorithm 1:
 *   collision detection -> hash-grid broadphase, particle-particle /
 *       particle-heightfield / particle-box contacts;
 *   the iterative PGS solve of the mesoscale MCP -> colour-sweep projected
 *       Gauss-Seidel on the contact law of Eqs. signCoul1-3 with the Hertz
 *       mapping and the SPOOK stepper (section "Contacting rigid
 *       multibodies");
 *   the position update x_{i+1} = x_i + dt v_{i+1}.
 *
 * Conventions
 *  - Every call returns a tds_status; nothing throws across the ABI.
 *    tds_last_error() gives a message for the calling thread.
 *  - Host pointers are caller-owned and only read (or written) during the
 *    call. Units are SI. Arrays are structure-of-arrays of float32 indexed by
 *    the particle id 0..n-1 given at creation.
 *  - Device memory is owned by the scene: either allocated by the library
 *    (workspace == NULL) or carved from one caller-provided device buffer of
 *    tds_workspace_bytes() bytes (for example a torch tensor); the caller then
 *    keeps it alive until tds_destroy_scene.
 *  - All device work of a scene is issued on one CUDA stream (the caller's,
 *    or the default stream when none is given). tds_step returns without
 *    waiting for the GPU; the read calls and tds_synchronize wait.
 *  - Errors detected on the device (capacity overflow, non-finite state,
 *    a grid barrier that timed out) are latched by the step that meets them
 *    and returned by the next waiting call (a read, tds_synchronize,
 *    tds_get_stats). That step and the steps queued after it change nothing,
 *    and the waiting call puts the scene back at the state before the failing
 *    step: particles, warm-start memory and heightfield as they were, the
 *    step count reduced accordingly (tds_get_stats). The scene is usable
 *    again; the call that reports the error leaves its output buffers
 *    unspecified. An error that no step raised leaves the scene unusable
 *    (TDS_ERR_STATE) until destroyed.
 *  - Not thread-safe per scene; distinct scenes may be used concurrently.
 */
#ifndef TDS_H
#define TDS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TDS_OK = 0,
  TDS_ERR_INVALID_ARG = -1,     /* a NULL, negative or inconsistent argument */
  TDS_ERR_CUDA = -2,            /* a CUDA runtime call failed (message says which) */
  TDS_ERR_OOM = -3,             /* device allocation failed or workspace too small */
  TDS_ERR_CAPACITY = -4,        /* more contacts or colours than the scene's capacity */
  TDS_ERR_NONFINITE = -5,       /* a particle velocity or position became NaN/Inf */
  TDS_ERR_BARRIER_TIMEOUT = -6, /* a grid-wide barrier waited longer than its limit */
  TDS_ERR_STATE = -7            /* the scene holds an error no step raised, or a call out of order */
} tds_status;

typedef enum { TDS_WARM_COLD = 0, TDS_WARM_PREV = 1, TDS_WARM_LEARNED = 2 } tds_warm_start;

/* Scene description. All pointers are host pointers, read during
 * tds_create_scene only.
 *
 * Particles (section "Particles"/"Mesoscale model", Eq. eqmotb): n spheres of
 *   radius r, density rho: m = rho 4/3 pi r^3, I = 2/5 m r^2.
 * Contact law (Eqs. signCoul1-3, Hertz mapping): Young's modulus E, Poisson
 *   ratio nu, friction mu_t (mu_tool against the tool), rolling resistance
 *   mu_r, particle cohesion c_p [Pa]. With c_p > 0 a contact exists while the
 *   gap is below delta_c = 0.025 (r_a + r_b) and can pull with an impulse of
 *   at most dt c_p pi rbar^2 (rbar = 2 r_a r_b / (r_a + r_b); r_a for walls
 *   and terrain; tool contacts have no cohesion).
 * Heightfield (Eq. surface, linearly interpolated): (hf_nx+1)*(hf_ny+1)
 *   heights h[j*(hf_nx+1)+i] at (hf_x0 + i*hf_cell, hf_y0 + j*hf_cell), each
 *   cell split into two triangles by the diagonal (i+1,j)-(i,j+1).
 *   hf_nx == 0 disables the terrain.
 * Walls: n_walls static boxes, 10 floats each: centre[3], unit quaternion
 *   (w,x,y,z)[4], half extents[3], in the world frame.
 * Tool: n_tool_boxes boxes in the tool frame (same 10-float layout); the
 *   tool's pose and velocity come from tds_set_tool_pose. At most
 *   TDS_MAX_BOXES walls + tool boxes in total.
 * Solver (SPOOK, tau_n = 2 dt; PGS): time step dt, gravity, sweeps per step
 *   (max_iters). tol > 0 switches to residual mode: stop when the
 *   diagonally scaled natural-map residual is <= tol, checked every
 *   residual_every sweeps, at most max_iters sweeps. residual_every = 0 checks
 *   adaptively: first after 5 sweeps, then where the residual's geometric
 *   decay between the last two checks predicts the tolerance (2 to 64 sweeps
 *   on); the criterion is the same, only the check schedule differs.
 * Capacity: contacts_per_particle (0 = 10) bounds the contact count by
 *   contacts_per_particle * n; exceeding it is TDS_ERR_CAPACITY.
 * Broadphase domain: particles are binned in a uniform grid over the box
 *   [domain_lo, domain_hi]; particles outside it still collide correctly
 *   (they fall into the border cells). A zero box lets the library choose it
 *   from the particles, heightfield and walls.
 */
#define TDS_MAX_BOXES 24
#define TDS_MAX_SCENES 4096  /* scenes in one batch */

typedef struct {
  uint32_t n;
  const float *x, *y, *z;      /* positions [m] */
  const float *vx, *vy, *vz;   /* velocities [m/s] (NULL: zero) */
  const float *wx, *wy, *wz;   /* angular velocities [rad/s] (NULL: zero) */
  const float *radius;         /* [m] */
  float density, young, poisson;
  float mu_t, mu_r, cohesion, mu_tool;
  uint32_t hf_nx, hf_ny;
  float hf_x0, hf_y0, hf_cell;
  const float *hf_heights;
  uint32_t n_walls;
  const float *walls;
  uint32_t n_tool_boxes;
  const float *tool_boxes;
  float dt, gravity[3];
  uint32_t max_iters;
  float tol;
  uint32_t residual_every;
  int32_t warm_start;          /* tds_warm_start */
  uint32_t contacts_per_particle;
  float domain_lo[3], domain_hi[3];
  /* Impact stage (the Newton impact law of section "Contacting rigid
   * multibodies"), a velocity-level solve before the main one: a contact whose
   * approach speed at the start of the step, -G_n v_n, exceeds impact_speed
   * gets the target G_n v+ = restitution * (-G_n v_n); every other normal row
   * is held at G_n v+ >= 0; friction and rolling keep their cones; no
   * cohesion; rigid rows, impulses from zero, impact_iters colour sweeps on the
   * predicted velocities; the main solve then starts from v+ (its q_n takes the
   * post-impact normal velocities). impact_iters == 0 disables it. The tool
   * force reports the main solve's impulses. */
  float restitution, impact_speed;
  uint32_t impact_iters;
} tds_scene_desc;

typedef struct tds_scene tds_scene; /* opaque */

typedef struct {
  uint32_t n_contacts, n_pp, n_static, n_colours, iterations;
  float residual;              /* natural-map residual of the final impulses */
  uint64_t steps;              /* steps taken since creation */
  uint64_t kernel_launches;    /* kernels launched since creation */
  uint32_t timed_steps;        /* steps timed since the previous tds_get_stats */
  float phase_ms[5];           /* summed over those steps: broadphase, narrowphase
                                  (contacts, rows, warm start), colouring, PGS solve,
                                  finish (write-back, tool force, integration) */
  /* sums over the steps since the previous tds_get_stats (which resets them):
     sweeps x particle-pair contacts, sweeps x static contacts, contacts, steps */
  uint64_t sweep_contacts_pp, sweep_contacts_static, sum_contacts, solved_steps;
  uint32_t colour_rounds;      /* rounds of the parallel greedy colouring, last step */
  uint32_t impacts;            /* contacts treated as impacts, last step */
  uint32_t spawned;            /* particles the active zones created, last step */
} tds_step_stats;

/* Bytes of device workspace a scene with this description needs. */
tds_status tds_workspace_bytes(const tds_scene_desc *desc, uint64_t *bytes);

/* Create a scene: validates desc, uploads the particle state and geometry.
 * workspace: NULL (the library allocates with cudaMalloc) or a device
 * pointer to at least tds_workspace_bytes() bytes, 256-byte aligned.
 * stream: a cudaStream_t, or NULL for the default stream. */
tds_status tds_create_scene(const tds_scene_desc *desc, void *workspace,
                            uint64_t workspace_bytes, void *stream, tds_scene **out);

/* Pose (position, unit quaternion w,x,y,z) and velocity (linear, angular,
 * world frame) of the kinematic tool for the following steps (Algorithm 1:
 * the equipment's state comes from the macroscale model). The pose is held
 * fixed during a step; its velocity enters the contact rows. */
tds_status tds_set_tool_pose(tds_scene *s, const float pos[3], const float quat[4],
                             const float linvel[3], const float angvel[3]);

/* Change the solver settings for the following steps: sweeps (or the cap in
 * residual mode), tol (> 0: residual mode) and the residual check period
 * (0: adaptive, see tds_scene_desc). */
tds_status tds_set_solver(tds_scene *s, uint32_t max_iters, float tol, uint32_t residual_every);

/* Change the impact stage (restitution, impact_speed, impact_iters; see
 * tds_scene_desc) for the following steps. */
tds_status tds_set_impact(tds_scene *s, float restitution, float impact_speed, uint32_t impact_iters);

/* Colouring of the contact graph (the order of the projected Gauss-Seidel
 * sweep): every period-th step (counting from the scene's first, step 0)
 * colours every contact greedily in hashed-priority order; the steps between
 * keep, for each contact whose key existed in the previous step, that step's
 * colour (two such contacts share a particle now iff they did then, so the
 * kept colours stay proper) and colour only the new contacts, each with the
 * smallest colour that no kept neighbour and no new neighbour of higher
 * priority uses. 1 (the default) colours every contact every step. The step
 * counter is that of tds_get_stats (restored with a checkpoint or a
 * rollback), so a scene's colourings do not depend on how its steps were
 * issued. */
tds_status tds_set_recolour_period(tds_scene *s, uint32_t period);

/* Change the warm start (tds_warm_start) for the following steps;
 * TDS_WARM_LEARNED needs tds_set_mlp_weights before the next step. */
tds_status tds_set_warm_start(tds_scene *s, int32_t mode);

/* Advance nsteps time steps (asynchronous). */
tds_status tds_step(tds_scene *s, uint32_t nsteps);

/* Wait for the scene's stream; returns a latched device error, if any (the
 * scene is then back at the state before the failing step). */
tds_status tds_synchronize(tds_scene *s);

/* Copy the particle state to host arrays of n floats (any pointer may be
 * NULL to skip it). n must equal the scene's particle count. Waits. */
tds_status tds_read_particles(tds_scene *s, float *x, float *y, float *z, float *vx,
                              float *vy, float *vz, float *wx, float *wy, float *wz,
                              uint32_t n);

/* Force [N] and torque about the tool origin [N m] exerted by the soil on the
 * tool during the last step (impulses / dt). Waits. */
tds_status tds_read_tool_force(tds_scene *s, float force[3], float torque[3]);

/* Contacts of the last step, at most cap of them, in no particular order:
 * key = (a << 32) | b for particles a < b, (a << 32) | 0x80000000 | s for
 * particle a against static surface s (0 heightfield, 1.. walls, then tool
 * boxes); lam = 7 floats per contact: normal impulse, tangent impulse
 * (world frame, 3), rolling impulse (3) [N s]; colour = its colour.
 * *count receives the total. Waits. */
tds_status tds_read_contacts(tds_scene *s, uint64_t *keys, float *lam, uint32_t *colour,
                             uint32_t cap, uint32_t *count);

/* Statistics of the last step (phase times: summed since the previous call,
 * which they reset). Waits. */
tds_status tds_get_stats(tds_scene *s, tds_step_stats *out);

/* Enable (1) or disable (0) per-phase timing with CUDA events recorded on the
 * scene's stream around each phase of every step. */
tds_status tds_set_timing(tds_scene *s, int32_t enable);

void tds_destroy_scene(tds_scene *s);

/* ---- batches of independent scenes ------------------------------------------
 * The paper runs one terrain per simulation; a batch advances several
 * independent terrain patches (for example the work sites of several
 * machines, or many training episodes) through the same launches of the
 * step above. Each scene keeps its own particles, heightfield, walls, tool
 * and friction coefficients (mu_t, mu_r, mu_tool); all scenes share dt,
 * gravity, density, young, poisson, cohesion, the solver settings,
 * warm_start and contacts_per_particle (creation fails otherwise). Scenes
 * never interact: every scene of a batch steps exactly as it would alone.
 * A batch is a tds_scene handle; the calls above apply to it as a whole:
 * particle ids are global, scene q owning ids [o_q, o_q + n_q) with o_q the
 * sum of the earlier scenes' n; tds_set_tool_pose and tds_read_tool_force
 * address scene 0; statistics are summed over the batch. In residual mode
 * every scene has its own residual (the natural-map residual of its own
 * contacts) and stops sweeping at the first check where it is <= tol, as it
 * would alone; the step ends when every scene has stopped (or at max_iters).
 * tds_get_stats then reports the most sweeps any scene did and the largest
 * final residual; tds_batch_read_solve gives each scene's. At most
 * TDS_MAX_SCENES scenes. tds_create_scene is a batch of one. */
tds_status tds_batch_workspace_bytes(const tds_scene_desc *descs, uint32_t count, uint64_t *bytes);
tds_status tds_create_batch(const tds_scene_desc *descs, uint32_t count, void *workspace,
                            uint64_t workspace_bytes, void *stream, tds_scene **out);

/* Tool pose of scene `scene` of the batch (as tds_set_tool_pose). */
tds_status tds_batch_set_tool_pose(tds_scene *s, uint32_t scene, const float pos[3],
                                   const float quat[4], const float linvel[3],
                                   const float angvel[3]);

/* Tool poses of all scenes in one call: 13 floats per scene (position 3,
 * quaternion w,x,y,z 4, linear velocity 3, angular velocity 3), count = the
 * number of scenes. Stops at the first invalid pose (earlier scenes keep
 * their new pose). */
tds_status tds_batch_set_tool_poses(tds_scene *s, const float *poses, uint32_t count);

/* Particle state of scene `scene` (n must equal its particle count; arrays
 * indexed by the scene-local id). Waits. */
tds_status tds_batch_read_particles(tds_scene *s, uint32_t scene, float *x, float *y, float *z,
                                    float *vx, float *vy, float *vz, float *wx, float *wy,
                                    float *wz, uint32_t n);

/* Force and torque on every scene's tool during the last step: 6 floats per
 * scene (fx, fy, fz, tx, ty, tz), count = the number of scenes. Waits. */
tds_status tds_batch_read_tool_forces(tds_scene *s, float *force_torque, uint32_t count);

/* Each scene's solve in the last step: its residual at its last check (the
 * check that stopped it, or the last sweep) and its sweeps; count = the
 * number of scenes, either pointer may be NULL. Waits. */
tds_status tds_batch_read_solve(tds_scene *s, float *residual, uint32_t *sweeps, uint32_t count);

/* Replay each step from a CUDA graph (1) or launch its kernels one by one
 * (0, the default). The graph is captured on the next step and captured
 * again whenever the warm start, recording or solver settings change; tool
 * poses need no capture. Results are identical either way. Needs a stream
 * created by the caller (not the legacy default stream). Per-phase timing
 * (tds_set_timing) works with graphs: the graph then carries the phase
 * events. */
tds_status tds_set_graph(tds_scene *s, int32_t enable);

/* ---- aggregate bodies ------------------------------------------------------------
 * The coupling of the particles to the macroscale model (section "Macroscale
 * model", Eqs. aggregate_mass to aggregate_rot_vel): the particles of each
 * active zone are lumped into one rigid body with
 *   M = sum m_a, x_A = sum m_a x_a / M, v_A = sum m_a v_a / M,
 *   I_A = sum m_a (|x_a - x_A|^2 delta - (x_a - x_A)(x_a - x_A)^T),
 *   omega_A = I_A^+ sum m_a (x_a - x_A) x v_a
 * (the printed inertia is read as the point-mass tensor about the centre of
 * mass; I_A^+ is the pseudo-inverse: no spin about an axis without inertia;
 * voxels with fluidized mass are not part of this library).
 * A zone is the intersection of 1..TDS_ZONE_MAX_PLANES half-spaces of one
 * scene: a particle of that scene is inside iff, for every plane,
 * (n_x x + n_y y) + n_z z <= d evaluated in FP32 in this order; it belongs to
 * the first zone (in the given order) that contains it. Computed from the
 * state after the last step on the scene's stream, accumulated in FP64.
 * Waits. */
#define TDS_MAX_ZONES 64
#define TDS_ZONE_MAX_PLANES 8
typedef struct {
  uint32_t scene;     /* scene of the batch (0 for a single scene) */
  uint32_t n_planes;  /* 1 .. TDS_ZONE_MAX_PLANES */
  float planes[TDS_ZONE_MAX_PLANES][4];  /* (n_x, n_y, n_z, d) */
} tds_zone;
typedef struct {
  uint32_t count;     /* particles in the zone (0: all fields zero) */
  uint32_t pad;
  double mass;        /* [kg] */
  double com[3];      /* [m] */
  double vel[3];      /* [m/s] */
  double omega[3];    /* [rad/s] */
  double inertia[6];  /* about com: xx, yy, zz, xy, xz, yz [kg m^2] */
} tds_aggregate;
tds_status tds_aggregate_bodies(tds_scene *s, const tds_zone *zones, uint32_t count, tds_aggregate *out);

/* ---- coarse-grained fields and fluidized-mass advection ---------------------------
 * Section "Coarse-graining" (Eq. cg_velocity) and the conserved advection of
 * fluidized mass (Eq. advection) on a voxel grid: voxel (i, j, k) has its
 * corner at origin + (i, j, k) l0 and index v = (k ny + j) nx + i; vector
 * fields are interleaved, 3 floats per voxel (x, y, z).
 * tds_coarse_grain samples, at voxel centres, rho = sum_a m_a zeta(x - x_a),
 * p = sum_a m_a v_a zeta(x - x_a) and u = p / rho (0 where rho = 0) for the
 * particles of scene grid->scene after the last step. kernel 0: zeta = 1/l0^3
 * on the voxel containing the particle centre (FP32 floor((x - o) / l0),
 * clamped to the grid: mass is preserved exactly); kernel 1: the Gaussian
 * (sqrt(2 pi) R)^-3 exp(-|x|^2 / 2R^2), truncated beyond 3R. rho (nvox
 * floats), p and u (3 nvox floats) are device pointers, overwritten;
 * asynchronous on the scene's stream (FP32 atomic accumulation).
 * tds_advect_fluid advances rho_f by one first-order upwind finite-volume
 * step of d rho_f/dt + div(rho_f u) = r_f in a closed grid: the face between
 * two voxels carries u_f rho_upwind (u_f the mean of their velocity
 * components normal to the face), boundary faces carry nothing, so the total
 * mass changes only by dt sum r_f (to rounding). Stable for
 * max |u| dt / l0 <= 1/3. u, rho_f, source (or NULL) and rho_out (not
 * aliasing rho_f) are device pointers; stream a cudaStream_t or NULL;
 * asynchronous. The paper's kinetic and contact stress fields are not
 * provided. */
typedef struct {
  float origin[3];  /* [m] */
  float l0;         /* voxel size [m] */
  uint32_t nx, ny, nz;
  uint32_t scene;   /* scene of a batch whose particles are sampled */
} tds_grid;
tds_status tds_coarse_grain(tds_scene *s, const tds_grid *grid, int32_t kernel, float R, float *rho, float *p,
                            float *u);
tds_status tds_advect_fluid(const tds_grid *grid, const float *u, const float *rho_f, const float *source,
                            float dt, float *rho_out, void *stream);

/* ---- active zone: cutting the terrain into particles ----------------------------
 * Section "Mesoscale model": a cutting edge moving through the terrain
 * carries a wedge-shaped active zone bounded by the separation plane (the
 * blade face), the failure plane from the edge to the free surface, rising
 * ahead of the blade at theta = pi/2 - (phi + beta)/2 above the horizontal
 * (Eq. failure_plane; phi the soil's internal friction angle, beta the
 * separation plane's inclination to the horizontal), and the ends of the edge;
 * the terrain it overlaps turns into particles.
 * After each step, for a scene with a cutter on its tool: every heightfield
 * node whose point on the failure plane lies within the edge's length and at
 * least spawn_radius ahead of the blade, and whose height is above it, is
 * lowered onto the failure plane; bank_density times the removed height times
 * the cell area becomes the node's pending mass. A node cut this step then
 * places particles of radius spawn_radius at rest in its liberated column
 * (from its height up to the highest it has been), j-th at
 * height + spawn_radius (1 + 2j), first fit: a position is taken when it
 * lies at least spawn_radius from the planes of the heightfield triangles
 * around the node (heights after the step's cut), no active particle overlaps
 * it (FP32 test) and the pending mass pays for a particle (particle density);
 * nodes in index order, each particle taking the
 * scene's next dormant slot (radius 0, in increasing id order). Mass that finds
 * no place or slot stays pending. Not modelled: fluidized mass, the reverse
 * conversion (deposition, gap filling). All in FP32 on the device, after the
 * position update, on the scene's stream.
 * Dormant slots: particles created with radius 0 are reserve slots (no
 * contacts, no gravity, no mass) that the cut fills; tds_read_radii tells them
 * apart. */
typedef struct {
  float edge[3];        /* a point of the cutting edge, tool frame [m] */
  float dir[3];         /* direction along the edge, tool frame (normalised) */
  float length;         /* edge length [m]; 0 removes the cutter */
  float normal[3];      /* separation-plane normal pointing ahead into the soil, tool frame */
  float phi;            /* internal friction angle of the soil [rad] */
  float bank_density;   /* mass density of the resting terrain [kg/m^3] */
  float spawn_radius;   /* radius of the new particles [m]: <= the largest radius at creation,
                           <= half the heightfield cell */
} tds_cutter;
tds_status tds_set_cutter(tds_scene *s, uint32_t scene, const tds_cutter *cutter);

/* The scene's current heightfield heights and pending (cut, not yet
 * particle) mass per node [kg], (hf_nx+1)*(hf_ny+1) floats each (either may
 * be NULL). Waits. */
tds_status tds_read_heightfield(tds_scene *s, uint32_t scene, float *heights, float *pending, uint32_t count);

/* Radii of all particles by id (0: a dormant slot). Waits. */
tds_status tds_read_radii(tds_scene *s, float *r, uint32_t n);

/* ---- checkpoint / resume ------------------------------------------------------
 * The state a step carries into the next, as one host buffer: particle
 * positions, radii, velocities and spins (in the library's slot order), the
 * warm-start memory of the last step, the heightfield with its pending mass
 * and highest heights, each scene's tool pose and the step count. A scene
 * created from the same descriptions (same particle count, contact capacity,
 * heightfields and scenes) that loads it continues exactly as the saved one
 * would have: the same steps give the same results bit for bit. Settings
 * (solver, warm-start mode and network weights, cutters, impact stage, launch
 * shapes, graph replay) are not part of the state: set them again.
 * tds_state_bytes: the buffer size. tds_save_state: waits for the scene's
 * stream and copies the state of the last completed step into buf (caller
 * owned, at least tds_state_bytes); a latched device error is returned
 * instead (and rolls the scene back, see above). tds_load_state: checks the
 * buffer's header (TDS_ERR_INVALID_ARG for another layout or a foreign
 * buffer), then replaces the scene's state; statistics and the contacts of
 * tds_read_contacts stay those of the scene's own last step. The layout: a
 * 32-byte header (magic "TDSS", version, particles, capacity, heights,
 * scenes, steps, warm-start flag), 13 floats of tool pose per scene, then the
 * device arrays in a fixed order. */
tds_status tds_state_bytes(tds_scene *s, uint64_t *bytes);
tds_status tds_save_state(tds_scene *s, void *buf, uint64_t bytes);
tds_status tds_load_state(tds_scene *s, const void *buf, uint64_t bytes);

/* ---- launch shapes ------------------------------------------------------------
 * Knobs of the GPU schedule (the paper, a CPU method, has none). Results do
 * not depend on them: every setting gives the same impulses and states bit
 * for bit. pgs_blocks: persistent solver CTAs (one per SM at most);
 * pgs_sync: between colours the solver either synchronises each CTA only
 * with the CTAs whose particles it can touch (1, the default) or all CTAs
 * with a grid barrier (0); colour_blocks: persistent colouring CTAs;
 * pgs_threads x pgs_per_thread: the solver CTA's threads and contacts per
 * thread, one of the compiled shapes 416x1 (the default, two CTAs per SM),
 * 768x1, 512x2, 640x2, 512x3 (one CTA per SM) and 256x1 (three CTAs per SM);
 * in each, the last warp stages the contact rows and the other threads solve
 * (both 0 keep the current shape).
 * max_pgs_blocks / max_colour_blocks (read only) are the co-resident limits
 * (max_pgs_blocks for the current solver shape; a shape change with
 * pgs_blocks 0 lowers the solver CTAs to the new shape's limit if needed).
 * wait_limit_us: how long [microseconds] any CTA of the step's persistent
 * kernels waits for other CTAs (a grid barrier, a neighbour's progress flag)
 * before it gives up: it latches TDS_ERR_BARRIER_TIMEOUT, every
 * CTA returns, and the next waiting call reports the error and rolls the
 * scene back (see the conventions above). Default 2 000 000 (2 s); a
 * healthy step never comes near it. A limit shorter than the waits of a
 * normal step makes the step fail that way (the rollback path can be
 * exercised without any fault).
 * tds_set_launch_config ignores the max fields; a zero pgs_blocks,
 * colour_blocks or wait_limit_us keeps the current value. */
typedef struct {
  int32_t pgs_blocks, pgs_sync, colour_blocks;
  int32_t max_pgs_blocks, max_colour_blocks;
  int32_t pgs_threads, pgs_per_thread;
  int32_t wait_limit_us;
} tds_launch_config;
tds_status tds_get_launch_config(tds_scene *s, tds_launch_config *out);
tds_status tds_set_launch_config(tds_scene *s, const tds_launch_config *cfg);

/* ---- learned warm start ------------------------------------------------------
 * Not in the paper, whose discussion proposes data-driven models trained on
 * resolved simulations as future work: a 10 -> 64 -> 64 -> 3 ReLU network
 * predicts each contact's initial normal and friction impulses; projected
 * Gauss-Seidel then solves as usual (it reaches the same residual; only the
 * sweep count changes). Inputs per contact (10): (J_n v*)/(|g| h),
 * overlap/(r_a + r_b), the previous step's normal, |tangent| and
 * slip-aligned tangent impulse over W, persisted (0/1), coordination numbers
 * of both particles, depth below the local surface / (r_a + r_b), contact
 * type (0 pair, 1 terrain or wall, 2 tool); W = |g| h / (1/m_a + 1/m_b),
 * v* = v_n + h g, s the unit tangential slip velocity at v* (below 1e-6 m/s:
 * unit n x e_k, e_k the axis least aligned with n), surface = largest z + r
 * in columns of f x f heightfield cells with f the smallest integer such that
 * f * cell >= 4 r_max. Outputs (3): Lambda_n/W, (Lambda_t . s)/W,
 * (Lambda_t . (n x s))/W. BF16 weights, FP32 accumulation (tensor cores).
 * Parameters: FP32 vector of tds_mlp_param_count() floats, row-major
 * W1[64][10], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]. */
uint32_t tds_mlp_param_count(void);

/* Weights used by a scene created with warm_start = TDS_WARM_LEARNED (host
 * FP32 parameters, copied). Waits. */
tds_status tds_set_mlp_weights(tds_scene *s, const float *params, uint32_t count);

/* Record training data: with recording on, every step keeps each contact's
 * features (at the start of the step) and targets (its final impulses in the
 * output units above). */
tds_status tds_set_recording(tds_scene *s, int32_t enable);

/* The last recorded step's samples in owner order: feat 10 floats, targ 3
 * floats and key (as in tds_read_contacts) per contact, at most cap of them;
 * *count receives the total. Host pointers (any may be NULL). Waits. */
tds_status tds_read_training_samples(tds_scene *s, float *feat, float *targ, uint64_t *keys,
                                     uint32_t cap, uint32_t *count);

/* Device-buffer network calls for training (all pointers device memory,
 * stream a cudaStream_t or NULL; asynchronous). workspace holds
 * tds_mlp_workspace_bytes() bytes (the packed BF16 weights).
 * tds_mlp_forward: Y[m][3] of X[m][10].
 * tds_mlp_loss_grad: loss = (1/(3m)) sum (y - T)^2 into *loss and its
 *   gradient with respect to params into grad (both overwritten).
 * tds_mlp_adam_step: Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected
 *   with the 1-based step) on the FP32 params with moments mom, vel; zeroes
 *   grad. */
tds_status tds_mlp_workspace_bytes(uint64_t *bytes);
tds_status tds_mlp_forward(const float *params, const float *X, uint32_t m, float *Y,
                           void *workspace, void *stream);
tds_status tds_mlp_loss_grad(const float *params, const float *X, const float *T, uint32_t m,
                             float *grad, float *loss, void *workspace, void *stream);
tds_status tds_mlp_adam_step(float *params, float *grad, float *mom, float *vel, uint32_t step,
                             float lr, void *stream);

/* ---- particle-pair contacts without any allocation -------------------------
 * The paper has no counterpart to this call; it serves callers that cannot
 * let a library allocate device memory: simulators stepping in a fixed-rate
 * real-time loop, where cudaMalloc/cudaFree can synchronize the device and
 * miss the frame, and applications whose device memory is owned by their own
 * fixed-budget pool. It runs the particle-pair part of tds_step's contact
 * search (sorted-cell broadphase and the same bit-exact FP32 predicate) on
 * caller buffers and keeps its intermediate arrays in one file-scope device
 * array of about 5.3 MB that every GPU loading the library holds until exit.
 *
 * x, y, z, radius: device pointers to n floats (particle i at index i);
 * cohesive != 0 adds the cohesive band 0.025 (r_a + r_b) to the reach.
 * keys: device pointer to cap uint64 slots; receives (a << 32) | b for every
 * touching pair a < b, in an order that depends only on the inputs (equal
 * inputs give the same array, element by element); count: device pointer to
 * one uint32 that receives the number of pairs (if it exceeds cap, only the
 * first cap keys of that same order were written). stream: a cudaStream_t or
 * NULL. Asynchronous: results are ready when the stream is.
 * n above TDS_NOALLOC_MAX_PARTICLES is rejected with TDS_ERR_CAPACITY; a CUDA
 * error left pending by an earlier call is reported as TDS_ERR_CUDA (and left
 * pending) before anything is launched.
 * Calls no cudaMalloc, cudaFree or allocating library routine. The first call
 * on a device looks up the scratch array's device address (with that device
 * current) and keeps it, so make it before any stream capture; the kept
 * address does not survive a reset of the device (cudaDeviceReset). All
 * calls share the array: calls whose GPU work overlaps race, so keep them on
 * one stream. */
#define TDS_NOALLOC_MAX_PARTICLES 65536
tds_status tds_find_pair_contacts_noalloc(const float *x, const float *y, const float *z,
                                          const float *radius, uint32_t n, int32_t cohesive,
                                          uint64_t *keys, uint32_t cap, uint32_t *count,
                                          void *stream);

/* Message of the last failed call on this thread ("" if none). */
const char *tds_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
