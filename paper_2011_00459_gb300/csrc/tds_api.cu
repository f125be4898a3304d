// tds_api.cu -- host side of the C ABI declared in include/tds.h: scene and
// batch creation with the workspace layout, per-scene geometry tables, the
// per-step orchestration of the kernels on the scene's stream (optionally
// replayed as CUDA graphs), and the read calls. A scene is a batch of one.
#include <cmath>
#include <math.h>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tds_internal.cuh"

// launchers (tds_contacts.cu, tds_colour.cu, tds_solve.cu, tds_mlp.cu)
int tds_launch_broadphase(const DevPtrs &d, const StepConsts &k, uint32_t ncells, cudaStream_t st);
int tds_launch_narrowphase(const DevPtrs &d, const StepConsts &k, int use_prev, cudaStream_t st);
int tds_launch_colouring(const DevPtrs &d, uint32_t n, uint32_t cap, int coop_blocks,
                         int coop_threads, cudaStream_t st);
int tds_launch_bucketing(const DevPtrs &d, uint32_t cap, cudaStream_t st);
int tds_launch_features(const DevPtrs &d, const StepConsts &k, int *surf, uint32_t ncols, uint32_t cap,
                        int compact, cudaStream_t st);
void tds_launch_learned(const DevPtrs &d, const void *packed, uint32_t cap, int compact, cudaStream_t st);
size_t tds_mlp_packed_bytes();
int tds_mlp_params();
void tds_mlp_pack(const float *params, void *packed, cudaStream_t st);
void tds_mlp_forward_launch(const void *packed, const float *X, uint32_t m, float *Y, cudaStream_t st);
cudaError_t tds_mlp_loss_grad_launch(const void *packed, const float *X, const float *T, uint32_t m,
                                     float *grad, float *loss, cudaStream_t st);
void tds_mlp_adam_launch(float *params, float *grad, float *mom, float *vel, uint32_t step, float lr,
                         cudaStream_t st);
int tds_launch_predict(const DevPtrs &d, const StepConsts &k, cudaStream_t st);
cudaError_t tds_launch_pgs(const DevPtrs &d, const StepConsts &k, uint32_t max_iters, float tol,
                           uint32_t every, int apply_warm, int blocks, int sync, int shape, cudaStream_t st);
int tds_pgs_shapes();
void tds_pgs_shape(int i, int *threads, int *per_thread);
cudaError_t tds_launch_impact(const DevPtrs &d, const StepConsts &k, float e, float vimp, uint32_t iters,
                              int blocks, cudaStream_t st);
int tds_launch_finish(const DevPtrs &d, const StepConsts &k, uint32_t cap, cudaStream_t st);
int tds_launch_cut(const DevPtrs &d, const StepConsts &k, float *heights, uint32_t nh, cudaStream_t st);
void tds_launch_stage(const DevPtrs &d, uint32_t n, cudaStream_t st);
int tds_pgs_setup();
int tds_pgs_occupancy(int i);
int tds_launch_aggregate(const DevPtrs &d, uint32_t n, const tds_zone *zones, uint32_t nz, uint8_t *zone_id,
                         double *sums, tds_aggregate *out, cudaStream_t st);
size_t tds_aggregate_sums_words();
int tds_launch_coarse_grain(const DevPtrs &d, uint32_t n, const tds_grid &g, int kernel, float R, float *rho,
                            float *p, float *u, cudaStream_t st);
bool tds_grid_valid(const tds_grid *g);
const void *tds_colour_kernel();

namespace {

thread_local std::string g_err;

tds_status fail(tds_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

#define CUDA_TRY(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(TDS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
  } while (0)

// Rotation matrix (row-major, world = R local) of a quaternion (w, x, y, z),
// normalised in FP64. Together with the composition in compose_boxes this is
// the box-geometry contract: FP64 evaluation in exactly this order, rounded to
// FP32 before the contact predicate reads it.
void quat_to_matrix(const float q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double s = 1.0 / std::sqrt(((w * w + x * x) + y * y) + z * z);
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

struct Carver {
  char *base;
  size_t off = 0;
  template <class T>
  T *take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += sizeof(T) * (count ? count : 1);
    return p;
  }
};

// Per-scene host data of a batch.
struct SceneHost {
  uint32_t off, n;                  // particle ids [off, off + n)
  std::vector<float> walls, tools;  // 10 floats per box
  bool has_cutter = false;
  tds_cutter cutter{};
  float pos[3] = {0, 0, 0}, quat[4] = {1, 0, 0, 0}, vel[3] = {0, 0, 0}, angvel[3] = {0, 0, 0};
};

struct Layout {
  uint32_t S = 0, n = 0, cap = 0, ncells = 0, ntiles = 0, nheights = 1, nboxes = 0, ncols = 0;
  float rmax = 0.f;
  int gnx = 1, gny = 1, gnz = 1;
  float cell = 1.f;
  std::vector<SceneGeo> geo;
};

struct Extra {  // workspace regions that are not kernel pointers of DevPtrs
  tds_zone *zones = nullptr;       // aggregate bodies: zones, per-particle zone, sums, results
  uint8_t *zone_id = nullptr;
  double *agg_sums = nullptr;
  tds_aggregate *agg_out = nullptr;
  float *heights = nullptr;
  SceneGeo *geo = nullptr;
  BoxF *boxes = nullptr;
  int *surf = nullptr;
  void *packed = nullptr;
  float *params = nullptr;
  float *targ = nullptr;
};

// What a captured step depends on besides device memory: the kernel
// arguments that the host settings select.
struct GraphKey {
  int use_prev = -1, warm = -1, recording = -1, timing = -1;
  int pgs_blocks = -1, pgs_sync = -1, pgs_shape = -1, colour_blocks = -1, cutter = -1;
  uint32_t max_iters = 0, every = 0, impact_iters = 0;
  float tol = -1.f, restitution = -1.f, impact_speed = -1.f;
  unsigned long long wait_ns = 0;
  uint32_t recolour = 0;
  bool operator==(const GraphKey &o) const {
    return use_prev == o.use_prev && warm == o.warm && recording == o.recording && timing == o.timing &&
           wait_ns == o.wait_ns && recolour == o.recolour &&
           pgs_blocks == o.pgs_blocks && pgs_sync == o.pgs_sync && pgs_shape == o.pgs_shape &&
           colour_blocks == o.colour_blocks &&
           max_iters == o.max_iters && every == o.every && tol == o.tol && impact_iters == o.impact_iters &&
           restitution == o.restitution && impact_speed == o.impact_speed && cutter == o.cutter;
  }
};

struct StepGraph {  // a captured step for one parity of the double buffers
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  GraphKey key;
  uint64_t launches = 0;
  cudaGraphNode_t ev_node[6] = {};  // phase-boundary event records (timing graphs)
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
};

}  // namespace

struct tds_scene {
  tds_scene_desc desc;  // the common settings (solver, material, step)
  Layout L;
  StepConsts k;
  DevPtrs d;
  cudaStream_t st = nullptr;
  void *mem = nullptr;
  bool owns = false;
  bool have_prev = false;
  std::vector<SceneHost> scenes;
  std::vector<BoxF> host_boxes;
  bool geo_dirty = true;
  int pgs_blocks = 1, colour_blocks = 1;
  int pgs_sync = 1;       // solver: 1 neighbour synchronisation, 0 grid barrier
  int pgs_shape = 0;      // solver CTA shape (index of the compiled shapes)
  bool any_cutter = false;
  int max_pgs_blocks = 1, max_colour_blocks = 1;
  int sms = 1;
  uint64_t steps = 0;
  tds_status latched = TDS_OK;
  uint64_t launches = 0;
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // 6 per timed step
  size_t ev_used = 0;
  Extra x;
  bool recording = false, have_weights = false;
  bool graph = false;
  StepGraph graphs[2];
  cudaEvent_t graph_ev[6] = {};  // placeholders captured into timing graphs
  uint32_t parity = 0;
};

namespace {

tds_status validate(const tds_scene_desc *d) {
  if (!d) return fail(TDS_ERR_INVALID_ARG, "desc is NULL");
  if (d->n == 0 || d->n >= 0x7FFFFFFFu) return fail(TDS_ERR_INVALID_ARG, "n must be in [1, 2^31)");
  if (!d->x || !d->y || !d->z || !d->radius) return fail(TDS_ERR_INVALID_ARG, "positions and radii are required");
  if (!(d->dt > 0.f)) return fail(TDS_ERR_INVALID_ARG, "dt must be > 0");
  if (!(d->density > 0.f) || !(d->young > 0.f) || !(d->poisson >= 0.f && d->poisson < 0.5f))
    return fail(TDS_ERR_INVALID_ARG, "density, young > 0 and 0 <= poisson < 0.5 required");
  if (d->mu_t < 0.f || d->mu_r < 0.f || d->cohesion < 0.f || d->mu_tool < 0.f)
    return fail(TDS_ERR_INVALID_ARG, "friction, rolling resistance and cohesion must be >= 0");
  if (d->n_walls + d->n_tool_boxes > TDS_MAX_BOXES)
    return fail(TDS_ERR_INVALID_ARG, "too many boxes (TDS_MAX_BOXES)");
  if ((d->n_walls && !d->walls) || (d->n_tool_boxes && !d->tool_boxes))
    return fail(TDS_ERR_INVALID_ARG, "box arrays missing");
  if (d->hf_nx > 0 && (d->hf_ny == 0 || !d->hf_heights || !(d->hf_cell > 0.f)))
    return fail(TDS_ERR_INVALID_ARG, "heightfield needs ny > 0, heights and cell > 0");
  if (d->max_iters == 0) return fail(TDS_ERR_INVALID_ARG, "max_iters must be >= 1");
  if (d->warm_start != TDS_WARM_COLD && d->warm_start != TDS_WARM_PREV && d->warm_start != TDS_WARM_LEARNED)
    return fail(TDS_ERR_INVALID_ARG, "warm_start must be TDS_WARM_COLD, TDS_WARM_PREV or TDS_WARM_LEARNED");
  if (!(d->restitution >= 0.f && d->restitution <= 1.f) || !(d->impact_speed >= 0.f) ||
      !std::isfinite(d->impact_speed))
    return fail(TDS_ERR_INVALID_ARG, "restitution must be in [0, 1] and impact_speed >= 0");
  for (uint32_t i = 0; i < d->n; ++i)
    if (!(d->radius[i] >= 0.f) || !std::isfinite(d->radius[i]) || !std::isfinite(d->x[i]) ||
        !std::isfinite(d->y[i]) || !std::isfinite(d->z[i]))
      return fail(TDS_ERR_INVALID_ARG, "radii must be >= 0 (0: dormant slot) and positions finite");
  return TDS_OK;
}

// Scenes of one batch share the step, material and solver settings.
tds_status validate_batch(const tds_scene_desc *descs, uint32_t count) {
  if (!descs || count == 0) return fail(TDS_ERR_INVALID_ARG, "descs is NULL or count is 0");
  if (count > TDS_MAX_SCENES) return fail(TDS_ERR_INVALID_ARG, "more than TDS_MAX_SCENES scenes in a batch");
  uint64_t total = 0;
  for (uint32_t s = 0; s < count; ++s) {
    tds_status v = validate(descs + s);
    if (v != TDS_OK) return v;
    total += descs[s].n;
    const tds_scene_desc &a = descs[0], &b = descs[s];
    if (a.dt != b.dt || a.gravity[0] != b.gravity[0] || a.gravity[1] != b.gravity[1] ||
        a.gravity[2] != b.gravity[2] || a.density != b.density || a.young != b.young ||
        a.poisson != b.poisson || a.cohesion != b.cohesion || a.max_iters != b.max_iters ||
        a.tol != b.tol || a.residual_every != b.residual_every || a.warm_start != b.warm_start ||
        a.contacts_per_particle != b.contacts_per_particle || a.restitution != b.restitution ||
        a.impact_speed != b.impact_speed || a.impact_iters != b.impact_iters)
      return fail(TDS_ERR_INVALID_ARG,
                  "scenes of a batch must share dt, gravity, density, young, poisson, cohesion, the "
                  "solver settings, warm_start, contacts_per_particle and the impact stage");
  }
  if (total >= 0x7FFFFFFFull) return fail(TDS_ERR_INVALID_ARG, "too many particles in the batch");
  bool active = false;
  for (uint32_t q = 0; q < count && !active; ++q)
    for (uint32_t i = 0; i < descs[q].n && !active; ++i) active = descs[q].radius[i] > 0.f;
  if (!active) return fail(TDS_ERR_INVALID_ARG, "at least one particle needs a radius > 0");
  return TDS_OK;
}

// Broadphase domain of one scene: the given box, or its particles and walls
// with a margin and headroom above.
void scene_domain(const tds_scene_desc *d, float cell, float lo[3], float hi[3]) {
  bool given = false;
  for (int a = 0; a < 3; ++a) given |= d->domain_hi[a] > d->domain_lo[a];
  if (given) {
    for (int a = 0; a < 3; ++a) { lo[a] = d->domain_lo[a]; hi[a] = d->domain_hi[a]; }
    return;
  }
  const float *xs[3] = {d->x, d->y, d->z};
  bool any = false;  // active particles only: dormant slots may sit anywhere
  for (uint32_t i = 0; i < d->n; ++i) {
    if (!(d->radius[i] > 0.f)) continue;
    for (int a = 0; a < 3; ++a) {
      lo[a] = any ? std::fmin(lo[a], xs[a][i]) : xs[a][i];
      hi[a] = any ? std::fmax(hi[a], xs[a][i]) : xs[a][i];
    }
    any = true;
  }
  if (!any) {  // no active particle yet: the heightfield's extent, or the origin
    lo[0] = d->hf_nx ? d->hf_x0 : 0.f;
    lo[1] = d->hf_nx ? d->hf_y0 : 0.f;
    hi[0] = d->hf_nx ? d->hf_x0 + d->hf_nx * d->hf_cell : 1.f;
    hi[1] = d->hf_nx ? d->hf_y0 + d->hf_ny * d->hf_cell : 1.f;
    lo[2] = 0.f;
    hi[2] = 1.f;
    if (d->hf_nx)
      for (uint32_t q = 0; q < (d->hf_nx + 1) * (d->hf_ny + 1); ++q) {
        lo[2] = std::fmin(lo[2], d->hf_heights[q]);
        hi[2] = std::fmax(hi[2], d->hf_heights[q] + 1.f);
      }
  }
  for (uint32_t w = 0; w < d->n_walls; ++w) {  // the walls bound the bed
    const float *b = d->walls + 10 * w;
    double R[9];
    quat_to_matrix(b + 3, R);
    for (int a = 0; a < 2; ++a) {
      double ext = std::fabs(R[3 * a]) * b[7] + std::fabs(R[3 * a + 1]) * b[8] + std::fabs(R[3 * a + 2]) * b[9];
      lo[a] = std::fmin(lo[a], (float)(b[a] - ext));
      hi[a] = std::fmax(hi[a], (float)(b[a] + ext));
    }
  }
  float margin = 2.0f * cell;
  for (int a = 0; a < 3; ++a) { lo[a] -= margin; hi[a] += margin; }
  hi[2] += 0.25f * (hi[2] - lo[2]);
}

Layout plan(const tds_scene_desc *descs, uint32_t S) {
  Layout L;
  L.S = S;
  uint64_t cap = 64;
  uint32_t per = descs[0].contacts_per_particle ? descs[0].contacts_per_particle : 10u;
  float rmax = 0.f;
  for (uint32_t s = 0; s < S; ++s) {
    L.n += descs[s].n;
    cap += (uint64_t)per * descs[s].n;
    for (uint32_t i = 0; i < descs[s].n; ++i) rmax = std::fmax(rmax, descs[s].radius[i]);
  }
  if (cap > 0x7FFFFFF0ull) cap = 0x7FFFFFF0ull;
  L.cap = (uint32_t)cap;
  L.rmax = rmax;
  L.ntiles = (L.cap + TDS_TILE - 1) / TDS_TILE;
  // cells wider than any reach (2 r_max plus the cohesive band), with margin
  L.cell = 2.0f * rmax * 1.025f * 1.02f;
  std::vector<float> lo(3 * S), hi(3 * S);
  for (;;) {
    int dims[3] = {1, 1, 1};
    for (uint32_t s = 0; s < S; ++s) {
      scene_domain(descs + s, L.cell, &lo[3 * s], &hi[3 * s]);
      for (int a = 0; a < 3; ++a) {
        int n = (int)std::ceil((hi[3 * s + a] - lo[3 * s + a]) / L.cell);
        dims[a] = std::max(dims[a], std::max(n, 1));
      }
    }
    uint64_t tot = (uint64_t)S * dims[0] * dims[1] * dims[2];
    if (tot <= (1ull << 26)) {
      L.gnx = dims[0]; L.gny = dims[1]; L.gnz = dims[2];
      L.ncells = (uint32_t)tot;
      break;
    }
    L.cell *= 1.25f;  // coarser cells keep the grid bounded; correctness is unaffected
  }
  L.geo.resize(S);
  uint32_t hoff = 0, boff = 0, coff = 0, pid0 = 0;
  for (uint32_t s = 0; s < S; ++s) {
    const tds_scene_desc &d = descs[s];
    SceneGeo &G = L.geo[s];
    std::memset(&G, 0, sizeof(G));
    for (int a = 0; a < 3; ++a) G.lo[a] = lo[3 * s + a];
    G.hf_nx = (int)d.hf_nx; G.hf_ny = (int)d.hf_ny;
    G.hf_x0 = d.hf_x0; G.hf_y0 = d.hf_y0; G.hf_cell = d.hf_cell;
    G.hf_off = hoff;
    if (d.hf_nx > 0) hoff += (d.hf_nx + 1) * (d.hf_ny + 1);
    G.box0 = boff;
    G.nbox = d.n_walls + d.n_tool_boxes;
    G.nwall = d.n_walls;
    boff += G.nbox;
    G.mu_t = d.mu_t; G.mu_tool = d.mu_tool; G.mu_r = d.mu_r;
    G.pid0 = pid0;
    G.npart = d.n;
    pid0 += d.n;
    // surface columns of the learned warm start: heightfield cells grouped
    // cf x cf, cf the smallest integer with cf * cell >= 4 r_max of the scene
    if (d.hf_nx > 0) {
      float rs = 0.f;
      for (uint32_t i = 0; i < d.n; ++i) rs = std::fmax(rs, d.radius[i]);
      int cf = (int)std::ceil(4.0 * (double)rs / (double)d.hf_cell);
      if (cf < 1) cf = 1;
      G.cf = cf;
      G.ncx = ((int)d.hf_nx + cf - 1) / cf;
      G.ncy = ((int)d.hf_ny + cf - 1) / cf;
      G.col_off = coff;
      coff += (uint32_t)(G.ncx * G.ncy);
    }
  }
  L.nheights = hoff ? hoff : 1;
  L.nboxes = boff;
  L.ncols = coff;
  return L;
}

size_t carve(Carver &c, const Layout &L, DevPtrs &d, Extra &x, int pgs_blocks) {
  const uint32_t n = L.n, cap = L.cap;
  d.pos = c.take<float4>(n); d.pv = c.take<float4>(2 * (size_t)n);
  d.pid = c.take<uint32_t>(n); d.sid = c.take<uint32_t>(n);
  d.pos2 = c.take<float4>(n); d.pv2 = c.take<float4>(2 * (size_t)n);
  d.pid2 = c.take<uint32_t>(n); d.sid2 = c.take<uint32_t>(n);
  d.cell_of = c.take<uint32_t>(n);
  d.cell_count = c.take<uint32_t>(L.ncells + 2);  // + the trailing cell of dormant slots
  d.cell_start = c.take<uint32_t>(L.ncells + 2);
  d.cell_cursor = c.take<uint32_t>(L.ncells + 1);
  d.perm = c.take<uint32_t>(n);
  d.cnt = c.take<uint32_t>(n + 1);
  d.cstart = c.take<uint32_t>(n + 1);
  d.c_ab = c.take<uint2>(cap);
  d.c_key = c.take<unsigned long long>(cap);
  d.c_rn = c.take<float4>(cap); d.c_rq = c.take<float4>(cap);
  d.c_rm = c.take<float2>(cap);
  d.c_sv = c.take<float4>(cap); d.c_sw = c.take<float4>(cap);
  d.c_la = c.take<float4>(cap); d.c_lb = c.take<float2>(cap);
  d.inc_cnt = c.take<uint32_t>(n + 1); d.inc_start = c.take<uint32_t>(n + 1);
  d.inc_cursor = c.take<uint32_t>(n); d.inc_ent = c.take<uint2>(2 * (size_t)cap);
  d.prio = c.take<unsigned long long>(cap);
  d.colour = c.take<uint8_t>(cap);
  d.wait = c.take<int32_t>(cap);
  d.frontier0 = c.take<uint32_t>(cap); d.frontier1 = c.take<uint32_t>(cap);
  d.ntiles = L.ntiles;
  d.tile_hist = c.take<uint32_t>((size_t)TDS_NBUCKETS * L.ntiles);
  d.tile_off = c.take<uint32_t>((size_t)TDS_NBUCKETS * L.ntiles + 1);
  d.bstart = c.take<uint32_t>(TDS_NBUCKETS + 1);
  d.bend = c.take<uint32_t>(TDS_NBUCKETS);
  d.bpad = c.take<uint32_t>(TDS_NBUCKETS);
  const size_t pc = (size_t)cap + TDS_ORDER_PAD;  // colour order with padding
  d.order = c.take<uint32_t>(pc);
  d.p_ab = c.take<uint2>(pc);
  d.p_rn = c.take<float4>(pc); d.p_rq = c.take<float4>(pc);
  d.p_rm = c.take<float2>(pc);
  d.p_sv = c.take<float4>(pc); d.p_sw = c.take<float4>(pc);
  d.p_la = c.take<float4>(pc); d.p_lb = c.take<float2>(pc);
  d.p_il = c.take<float4>(pc); d.p_il2 = c.take<float4>(pc);
  for (int b = 0; b < 2; ++b) {
    d.prev_first[b] = c.take<uint32_t>(n);
    d.prev_cnt[b] = c.take<uint32_t>(n);
    d.prev_other[b] = c.take<uint32_t>(cap);
    d.prev_l0[b] = c.take<float4>(cap);
    d.prev_l1[b] = c.take<float4>(cap);
  }
  d.err = c.take<int32_t>(1);
  d.ctr = c.take<uint32_t>(CTR_COUNT);
  d.acc = c.take<unsigned long long>(ACC_COUNT);
  d.fscal = c.take<float>(FS_COUNT);
  size_t nd = 2 * (size_t)pgs_blocks;
  if (nd < 6 * 128) nd = 6 * 128;
  d.dpart = c.take<double>(nd);
  const size_t nsb = (size_t)L.S * TDS_NBUCKETS;
  const size_t max_chunks = (size_t)cap / TDS_RES_CHUNK + nsb + 1;
  d.dres = c.take<double>(2 * max_chunks);
  d.nscenes = L.S;
  d.scq_cnt = c.take<uint32_t>(nsb);
  d.scq_start = c.take<uint32_t>(nsb);
  d.scq_chunk = c.take<uint32_t>(nsb + 1);
  d.chunk = c.take<uint4>(max_chunks);
  d.scene_res = c.take<float>(L.S);
  d.scene_iters = c.take<uint32_t>(L.S);
  d.bar = c.take<uint32_t>(2);
  d.prog = c.take<uint32_t>(kProgStride * (size_t)pgs_blocks);
  d.rng = c.take<uint32_t>(2 * (size_t)pgs_blocks);
  size_t m = L.ncells + 1;
  if (m < n) m = n;
  if (m < (size_t)TDS_NBUCKETS * L.ntiles) m = (size_t)TDS_NBUCKETS * L.ntiles;
  if (m < (size_t)L.nheights) m = L.nheights;
  d.scan_tmp = c.take<uint32_t>(tds_scan_tmp_words((uint32_t)m));
  d.stage = c.take<float>(10 * (size_t)n);
  d.tool_out = c.take<float>(6 * (size_t)L.S);
  d.tool_acc = c.take<double>(6 * (size_t)L.S);
  d.feat = c.take<float>(10 * (size_t)cap);
  d.sdirw = c.take<float4>(cap);
  d.c_flag = c.take<uint8_t>(cap);
  d.new_idx = c.take<uint32_t>(cap);
  d.hf_pend = c.take<float>(L.nheights);
  d.hf_top = c.take<float>(L.nheights);
  d.hf_scene = c.take<uint32_t>(L.nheights);
  d.hf_cnt = c.take<uint32_t>((size_t)L.nheights + 1);
  d.hf_rank = c.take<uint32_t>((size_t)L.nheights + 1);
  d.dorm_rank = c.take<uint32_t>((size_t)n + 1);
  d.dorm_list = c.take<uint32_t>(n);
  d.slot_of_pid = c.take<uint32_t>(n);
  x.targ = c.take<float>(3 * (size_t)cap);
  x.surf = c.take<int>(L.ncols);
  x.packed = c.take<unsigned char>(tds_mlp_packed_bytes());
  x.params = c.take<float>(tds_mlp_params());
  x.heights = c.take<float>(L.nheights);
  x.zones = c.take<tds_zone>(TDS_MAX_ZONES);
  x.zone_id = c.take<uint8_t>(n);
  x.agg_sums = c.take<double>(tds_aggregate_sums_words());
  x.agg_out = c.take<tds_aggregate>(TDS_MAX_ZONES);
  x.geo = c.take<SceneGeo>(L.S);
  x.boxes = c.take<BoxF>(L.nboxes);
  return c.off + 256;
}

int pgs_blocks_for(uint32_t n, int max_coop) {
  int b = (int)((n + 511) / 512);
  if (b < 1) b = 1;
  return b < max_coop ? b : max_coop;
}

void set_box(BoxF &B, const double R[9], const double c[3], const float h[3], int is_tool) {
  for (int i = 0; i < 9; ++i) B.R[i] = (float)R[i];
  for (int i = 0; i < 3; ++i) { B.c[i] = (float)c[i]; B.h[i] = h[i]; }
  B.is_tool = is_tool;
}

double norm3d(const double a[3]) { return std::sqrt((a[0] * a[0] + a[1] * a[1]) + a[2] * a[2]); }

// The active-zone wedge of scene s's cutter on the tool pose (rotation RT),
// in FP64 then rounded: edge start e0 = p_T + R_T edge, edge direction u and
// blade normal ns (normalised), beta = the separation plane's inclination to
// the horizontal = acos |ns_z|, theta = pi/2 - (phi + beta)/2 (Eq.
// failure_plane), the failure plane through the edge spanned by u and
// d = (cos theta f, sin theta) with f the horizontal direction of ns; its
// normal nf = d x u points up.
void compose_wedge(tds_scene *S, uint32_t s, const double RT[9]) {
  const SceneHost &h = S->scenes[s];
  SceneGeo &G = S->L.geo[s];
  G.cut_on = 0;
  if (!h.has_cutter || !(h.cutter.length > 0.f)) return;
  const tds_cutter &c = h.cutter;
  double e[3], u[3], ns[3];
  for (int i = 0; i < 3; ++i) {
    e[i] = (double)h.pos[i] + ((RT[3 * i] * (double)c.edge[0] + RT[3 * i + 1] * (double)c.edge[1]) +
                               RT[3 * i + 2] * (double)c.edge[2]);
    u[i] = (RT[3 * i] * (double)c.dir[0] + RT[3 * i + 1] * (double)c.dir[1]) + RT[3 * i + 2] * (double)c.dir[2];
    ns[i] = (RT[3 * i] * (double)c.normal[0] + RT[3 * i + 1] * (double)c.normal[1]) +
            RT[3 * i + 2] * (double)c.normal[2];
  }
  const double lu = norm3d(u), ln = norm3d(ns);
  for (int i = 0; i < 3; ++i) { u[i] /= lu; ns[i] /= ln; }
  const double beta = std::acos(std::fmin(1.0, std::fabs(ns[2])));
  const double theta = 0.5 * M_PI - 0.5 * ((double)c.phi + beta);
  const double fh = std::sqrt(ns[0] * ns[0] + ns[1] * ns[1]);
  if (fh < 1e-9) return;
  const double f[2] = {ns[0] / fh, ns[1] / fh};
  const double dd[3] = {std::cos(theta) * f[0], std::cos(theta) * f[1], std::sin(theta)};
  double nf[3] = {dd[1] * u[2] - dd[2] * u[1], dd[2] * u[0] - dd[0] * u[2], dd[0] * u[1] - dd[1] * u[0]};
  if (nf[2] < 0.0) for (int i = 0; i < 3; ++i) nf[i] = -nf[i];
  const double lf = norm3d(nf);
  for (int i = 0; i < 3; ++i) nf[i] /= lf;
  if (std::fabs(nf[2]) < 1e-6) return;
  const double rs = (double)c.spawn_radius;
  const double m = S->desc.density * 4.0 / 3.0 * M_PI * rs * rs * rs;
  for (int i = 0; i < 3; ++i) {
    G.e0[i] = (float)e[i];
    G.u[i] = (float)u[i];
    G.ns[i] = (float)ns[i];
    G.nf[i] = (float)nf[i];
  }
  G.cut_len = c.length;
  G.rho_b = c.bank_density;
  G.rs = c.spawn_radius;
  G.ms = (float)m;
  G.inv_m = (float)(1.0 / m);
  G.inv_I = (float)(1.0 / (0.4 * m * rs * rs));
  G.cut_on = 1;
}

// World-frame boxes of scene s for its current tool pose: walls as given,
// tool boxes composed as R_w = R_T R_k, c_w = p_T + R_T c_k in FP64, then
// rounded; the tool motion goes to the scene's table entry.
void compose_boxes(tds_scene *S, uint32_t s) {
  const SceneHost &h = S->scenes[s];
  SceneGeo &G = S->L.geo[s];
  BoxF *out = S->host_boxes.data() + G.box0;
  const uint32_t nw = G.nwall, nt = G.nbox - G.nwall;
  for (uint32_t w = 0; w < nw; ++w) {
    const float *b = h.walls.data() + 10 * w;
    double R[9], c[3] = {b[0], b[1], b[2]};
    quat_to_matrix(b + 3, R);
    set_box(out[w], R, c, b + 7, 0);
  }
  double RT[9];
  quat_to_matrix(h.quat, RT);
  for (uint32_t t = 0; t < nt; ++t) {
    const float *b = h.tools.data() + 10 * t;
    double Rk[9], Rw[9], c[3];
    quat_to_matrix(b + 3, Rk);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        Rw[3 * i + j] = (RT[3 * i + 0] * Rk[0 + j] + RT[3 * i + 1] * Rk[3 + j]) + RT[3 * i + 2] * Rk[6 + j];
    for (int i = 0; i < 3; ++i) {
      double o = (RT[3 * i + 0] * (double)b[0] + RT[3 * i + 1] * (double)b[1]) + RT[3 * i + 2] * (double)b[2];
      c[i] = (double)h.pos[i] + o;
    }
    set_box(out[nw + t], Rw, c, b + 7, 1);
  }
  for (int i = 0; i < 3; ++i) {
    G.tp[i] = h.pos[i];
    G.tv[i] = h.vel[i];
    G.tw[i] = h.angvel[i];
  }
  compose_wedge(S, s, RT);
  S->geo_dirty = true;
}

tds_status check_latched(tds_scene *s) {
  if (s->latched != TDS_OK) return fail(TDS_ERR_STATE, "scene holds an earlier error");
  return TDS_OK;
}

const char *dev_err_text(int32_t e) {
  switch (e) {
    case DEV_ERR_CAPACITY: return "contact or colour capacity exceeded (raise contacts_per_particle)";
    case DEV_ERR_NONFINITE: return "non-finite particle state";
    case DEV_ERR_BARRIER: return "grid barrier wait exceeded its time limit";
    default: return "device error";
  }
}

// The buffers one step swaps: particle state (sorted copy / previous order)
// and warm-start memory (read / written this step).
void swap_state(DevPtrs &d) {
  std::swap(d.pos, d.pos2);
  std::swap(d.pv, d.pv2);
  std::swap(d.pid, d.pid2);
  std::swap(d.sid, d.sid2);
  std::swap(d.prev_first[0], d.prev_first[1]);
  std::swap(d.prev_cnt[0], d.prev_cnt[1]);
  std::swap(d.prev_other[0], d.prev_other[1]);
  std::swap(d.prev_l0[0], d.prev_l0[1]);
  std::swap(d.prev_l1[0], d.prev_l1[1]);
}

// Waits for the scene's stream and reports a latched device error. A failing
// step leaves the scene as it was before that step: the error was latched in
// the last step that started clean (CTR_CLEAN counts them), no kernel wrote
// state after it, and that step's input still sits in the buffers the step
// swapped away from. Restoring their parity (and clearing the error) makes
// the scene usable again; the call returns the error.
tds_status sync_and_check(tds_scene *s) {
  CUDA_TRY(cudaStreamSynchronize(s->st));
  int32_t e = 0;
  CUDA_TRY(cudaMemcpy(&e, s->d.err, sizeof(e), cudaMemcpyDeviceToHost));
  if (e != 0) {
    uint32_t clean = 0;
    CUDA_TRY(cudaMemcpy(&clean, s->d.ctr + CTR_CLEAN, sizeof(clean), cudaMemcpyDeviceToHost));
    if (clean == 0 || clean > s->steps) {  // not raised by a step: keep it
      s->latched = (tds_status)e;
      return fail((tds_status)e, dev_err_text(e));
    }
    const uint64_t keep = clean - 1u;  // steps that completed
    if ((s->steps - keep) & 1u) {
      swap_state(s->d);
      s->parity ^= 1u;
    }
    s->steps = keep;
    s->have_prev = keep > 0;
    const int32_t zero = 0;
    const uint32_t k32 = (uint32_t)keep;
    CUDA_TRY(cudaMemcpy(s->d.err, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(s->d.ctr + CTR_CLEAN, &k32, sizeof(k32), cudaMemcpyHostToDevice));
    return fail((tds_status)e, std::string(dev_err_text(e)) + " in step " + std::to_string(clean) +
                                   "; the scene is back at the state before that step");
  }
  return TDS_OK;
}

tds_status workspace_bytes_impl(const tds_scene_desc *descs, uint32_t count, uint64_t *bytes) {
  tds_status v = validate_batch(descs, count);
  if (v != TDS_OK) return v;
  if (!bytes) return fail(TDS_ERR_INVALID_ARG, "bytes is NULL");
  Layout L = plan(descs, count);
  DevPtrs d{};
  Extra x;
  Carver c{nullptr};
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *bytes = carve(c, L, d, x, 64 * sms);
  return TDS_OK;
}

tds_status create_impl(const tds_scene_desc *descs, uint32_t count, void *workspace, uint64_t workspace_bytes,
                       void *stream, tds_scene **out) {
  tds_status v = validate_batch(descs, count);
  if (v != TDS_OK) return v;
  if (!out) return fail(TDS_ERR_INVALID_ARG, "out is NULL");
  if (workspace && ((uintptr_t)workspace & 255u))
    return fail(TDS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  *out = nullptr;
  tds_scene *s = new tds_scene();
  s->desc = descs[0];
  s->st = (cudaStream_t)stream;
  s->L = plan(descs, count);
  s->scenes.resize(count);
  uint32_t off = 0;
  for (uint32_t q = 0; q < count; ++q) {
    SceneHost &h = s->scenes[q];
    h.off = off;
    h.n = descs[q].n;
    off += h.n;
    if (descs[q].n_walls) h.walls.assign(descs[q].walls, descs[q].walls + 10 * descs[q].n_walls);
    if (descs[q].n_tool_boxes)
      h.tools.assign(descs[q].tool_boxes, descs[q].tool_boxes + 10 * descs[q].n_tool_boxes);
  }
  int dev = 0, sms = 0, occ_pgs = 0, occ_col = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (ce == cudaSuccess) occ_pgs = tds_pgs_setup();
  if (ce == cudaSuccess) ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_col, tds_colour_kernel(), 256, 0);
  if (ce != cudaSuccess || occ_pgs < 1 || occ_col < 1) {
    delete s;
    if (ce == cudaSuccess)
      return fail(TDS_ERR_CUDA, "a solver or colouring CTA shape does not fit on one SM (shared memory or "
                                "registers)");
    return fail(TDS_ERR_CUDA, std::string("device query failed: ") + cudaGetErrorString(ce));
  }
  s->sms = sms;
  // the default solver shape's co-resident CTAs at most
  s->pgs_blocks = pgs_blocks_for(s->L.n, sms * std::max(1, tds_pgs_occupancy(0)));
  s->colour_blocks = sms * (occ_col < 4 ? occ_col : 4);
  s->max_pgs_blocks = 64 * sms;  // the workspace's limit; each shape's co-residency limits it further
  s->max_colour_blocks = sms * occ_col;
  Carver probe{nullptr};
  DevPtrs tmp{};
  Extra tx;
  size_t need = carve(probe, s->L, tmp, tx, 64 * sms);
  if (workspace) {
    if (workspace_bytes < need) {
      delete s;
      return fail(TDS_ERR_OOM, "workspace smaller than tds_workspace_bytes()");
    }
    s->mem = workspace;
  } else {
    if (cudaMalloc(&s->mem, need) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return fail(TDS_ERR_OOM, "cudaMalloc of the scene workspace failed");
    }
    s->owns = true;
  }
  Carver c{(char *)s->mem};
  carve(c, s->L, s->d, s->x, 64 * sms);
  s->d.targ = nullptr;
  s->d.wait_ns = TDS_BARRIER_NS;
  s->d.recolour = 1u;
  // common constants
  const tds_scene_desc &D = descs[0];
  StepConsts &k = s->k;
  std::memset(&k, 0, sizeof(k));
  k.n = s->L.n;
  k.cap = s->L.cap;
  k.nscenes = count;
  k.dt = D.dt;
  for (int i = 0; i < 3; ++i) k.g[i] = D.gravity[i];
  k.ups = 1.0f / (1.0f + 4.0f * (2.0f * D.dt) / D.dt);
  double nu = D.poisson, E = D.young;
  k.estar_pair = (float)(1.0 / (2.0 * (1.0 - nu * nu) / E));
  k.estar_static = (float)(E / (1.0 - nu * nu));
  k.cohesion = D.cohesion;
  k.cohesive = D.cohesion > 0.f;
  k.sig_t = 1e-9f / D.dt;
  k.sig_r = 1e-9f / D.dt;
  k.cell_inv = 1.0f / s->L.cell;
  k.gnx = s->L.gnx; k.gny = s->L.gny; k.gnz = s->L.gnz;
  k.geo = s->x.geo;
  k.boxes = s->x.boxes;
  k.heights = s->x.heights;
  s->host_boxes.resize(s->L.nboxes);
  for (uint32_t q = 0; q < count; ++q) compose_boxes(s, q);
  // particle state: (x, r), (v, 1/m | w, 1/I), ids, scenes
  const uint32_t n = s->L.n;
  std::vector<float4> P(n), PV(2 * (size_t)n);
  std::vector<uint32_t> ids(n), sids(n);
  std::vector<float> heights(s->L.nheights, 0.f);
  const double pi = 3.14159265358979323846;
  for (uint32_t q = 0; q < count; ++q) {
    const tds_scene_desc &d = descs[q];
    const uint32_t o = s->scenes[q].off;
    for (uint32_t i = 0; i < d.n; ++i) {
      double r = d.radius[i];
      P[o + i] = make_float4(d.x[i], d.y[i], d.z[i], d.radius[i]);
      if (!(r > 0.0)) {  // dormant reserve slot: at rest, no mass (1/m = 1/I = 0)
        PV[2 * (size_t)(o + i)] = make_float4(0.f, 0.f, 0.f, 0.f);
        PV[2 * (size_t)(o + i) + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        double m = d.density * 4.0 / 3.0 * pi * r * r * r;
        double I = 0.4 * m * r * r;
        PV[2 * (size_t)(o + i)] = make_float4(d.vx ? d.vx[i] : 0.f, d.vy ? d.vy[i] : 0.f,
                                              d.vz ? d.vz[i] : 0.f, (float)(1.0 / m));
        PV[2 * (size_t)(o + i) + 1] = make_float4(d.wx ? d.wx[i] : 0.f, d.wy ? d.wy[i] : 0.f,
                                                  d.wz ? d.wz[i] : 0.f, (float)(1.0 / I));
      }
      ids[o + i] = o + i;
      sids[o + i] = q;
    }
    if (d.hf_nx > 0)
      std::memcpy(heights.data() + s->L.geo[q].hf_off, d.hf_heights,
                  sizeof(float) * (d.hf_nx + 1) * (d.hf_ny + 1));
  }
  std::vector<uint32_t> hf_scene(s->L.nheights, 0u);
  for (uint32_t q = 0; q < count; ++q)
    if (descs[q].hf_nx > 0)
      for (uint32_t k2 = 0; k2 < (descs[q].hf_nx + 1) * (descs[q].hf_ny + 1); ++k2)
        hf_scene[s->L.geo[q].hf_off + k2] = q;
  if (cudaMemcpyAsync(s->d.hf_scene, hf_scene.data(), sizeof(uint32_t) * hf_scene.size(), cudaMemcpyHostToDevice,
                      s->st) ||
      cudaMemcpyAsync(s->d.hf_top, heights.data(), sizeof(float) * heights.size(), cudaMemcpyHostToDevice, s->st) ||
      cudaMemsetAsync(s->d.hf_pend, 0, sizeof(float) * heights.size(), s->st) ||
      cudaMemcpyAsync(s->d.pos, P.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, s->st) ||
      cudaMemcpyAsync(s->d.pv, PV.data(), sizeof(float4) * 2 * n, cudaMemcpyHostToDevice, s->st) ||
      cudaMemcpyAsync(s->d.pid, ids.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s->st) ||
      cudaMemcpyAsync(s->d.sid, sids.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s->st) ||
      cudaMemcpyAsync(s->x.heights, heights.data(), sizeof(float) * heights.size(), cudaMemcpyHostToDevice,
                      s->st) ||
      cudaMemsetAsync(s->d.err, 0, sizeof(int32_t), s->st) ||
      cudaMemsetAsync(s->d.ctr, 0, sizeof(uint32_t) * CTR_COUNT, s->st) ||
      cudaMemsetAsync(s->d.acc, 0, sizeof(unsigned long long) * ACC_COUNT, s->st) ||
      cudaMemsetAsync(s->d.fscal, 0, sizeof(float) * FS_COUNT, s->st) ||
      cudaMemsetAsync(s->d.tool_out, 0, sizeof(float) * 6 * count, s->st) ||
      cudaMemsetAsync(s->d.tool_acc, 0, sizeof(double) * 6 * count, s->st) ||
      cudaMemsetAsync(s->d.bstart, 0, sizeof(uint32_t) * (TDS_NBUCKETS + 1), s->st) ||
      cudaMemsetAsync(s->d.bend, 0, sizeof(uint32_t) * TDS_NBUCKETS, s->st) ||
      cudaStreamSynchronize(s->st)) {
    cudaGetLastError();
    if (s->owns) cudaFree(s->mem);
    delete s;
    return fail(TDS_ERR_CUDA, "uploading the scene failed");
  }
  *out = s;
  return TDS_OK;
}

tds_status set_pose_impl(tds_scene *s, uint32_t q, const float pos[3], const float quat[4],
                         const float linvel[3], const float angvel[3]) {
  if (!s || !pos || !quat || !linvel || !angvel) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (q >= s->scenes.size()) return fail(TDS_ERR_INVALID_ARG, "scene index out of range");
  double qn = std::sqrt((double)quat[0] * quat[0] + (double)quat[1] * quat[1] +
                        (double)quat[2] * quat[2] + (double)quat[3] * quat[3]);
  if (!(qn > 1e-6)) return fail(TDS_ERR_INVALID_ARG, "quaternion has zero norm");
  SceneHost &h = s->scenes[q];
  for (int i = 0; i < 3; ++i) {
    if (!std::isfinite(pos[i]) || !std::isfinite(linvel[i]) || !std::isfinite(angvel[i]))
      return fail(TDS_ERR_INVALID_ARG, "non-finite tool pose");
    h.pos[i] = pos[i];
    h.vel[i] = linvel[i];
    h.angvel[i] = angvel[i];
  }
  for (int i = 0; i < 4; ++i) h.quat[i] = quat[i];
  compose_boxes(s, q);
  return TDS_OK;
}

// The kernels of one step, in order, on the scene's stream (capturable:
// under capture the phase events become event-record nodes of the graph).
tds_status enqueue_step(tds_scene *s, cudaEvent_t *E, uint64_t &launches, bool capture = false) {
  DevPtrs &d = s->d;
  const tds_scene_desc &D = s->desc;
  const unsigned evf = capture ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (E) CUDA_TRY(cudaEventRecordWithFlags(E[0], s->st, evf));
  launches += tds_launch_broadphase(d, s->k, s->L.ncells, s->st);
  std::swap(d.pos, d.pos2);
  std::swap(d.pv, d.pv2);
  std::swap(d.pid, d.pid2);
  std::swap(d.sid, d.sid2);
  if (E) CUDA_TRY(cudaEventRecordWithFlags(E[1], s->st, evf));
  const bool learned = D.warm_start == TDS_WARM_LEARNED;
  // the learned warm start also reads the previous step's impulses
  int use_prev = (D.warm_start != TDS_WARM_COLD) && s->have_prev;
  launches += tds_launch_narrowphase(d, s->k, use_prev, s->st);
  launches += tds_launch_predict(d, s->k, s->st);
  if (E) CUDA_TRY(cudaEventRecordWithFlags(E[2], s->st, evf));
  launches += tds_launch_colouring(d, s->L.n, s->L.cap, s->colour_blocks, 256, s->st);
  d.targ = s->recording ? s->x.targ : nullptr;
  // without recording the network needs the features of the new contacts only
  const int compact = learned && !s->recording;
  if (learned || s->recording)
    launches += tds_launch_features(d, s->k, s->x.surf, s->L.ncols, s->L.cap, compact, s->st);
  if (learned) {
    tds_launch_learned(d, s->x.packed, s->L.cap, compact, s->st);
    launches += 1;
  }
  launches += tds_launch_bucketing(d, s->L.cap, s->st);
  if (D.impact_iters > 0) {
    CUDA_TRY(tds_launch_impact(d, s->k, D.restitution, D.impact_speed, D.impact_iters, s->pgs_blocks, s->st));
    launches += 1;
  }
  if (E) CUDA_TRY(cudaEventRecordWithFlags(E[3], s->st, evf));
  CUDA_TRY(tds_launch_pgs(d, s->k, D.max_iters, D.tol, D.residual_every, use_prev || learned, s->pgs_blocks,
                          s->pgs_sync, s->pgs_shape, s->st));
  launches += 1;
  if (E) CUDA_TRY(cudaEventRecordWithFlags(E[4], s->st, evf));
  launches += tds_launch_finish(d, s->k, s->L.cap, s->st);
  if (s->any_cutter) launches += tds_launch_cut(d, s->k, s->x.heights, s->L.nheights, s->st);
  if (E) CUDA_TRY(cudaEventRecordWithFlags(E[5], s->st, evf));
  std::swap(d.prev_first[0], d.prev_first[1]);
  std::swap(d.prev_cnt[0], d.prev_cnt[1]);
  std::swap(d.prev_other[0], d.prev_other[1]);
  std::swap(d.prev_l0[0], d.prev_l0[1]);
  std::swap(d.prev_l1[0], d.prev_l1[1]);
  return TDS_OK;
}

GraphKey graph_key(const tds_scene *s) {
  GraphKey g;
  g.use_prev = (s->desc.warm_start != TDS_WARM_COLD) && s->have_prev;
  g.warm = s->desc.warm_start;
  g.recording = s->recording;
  g.max_iters = s->desc.max_iters;
  g.every = s->desc.residual_every;
  g.tol = s->desc.tol;
  g.timing = s->timing;
  g.pgs_blocks = s->pgs_blocks;
  g.pgs_sync = s->pgs_sync;
  g.pgs_shape = s->pgs_shape;
  g.colour_blocks = s->colour_blocks;
  g.impact_iters = s->desc.impact_iters;
  g.restitution = s->desc.restitution;
  g.impact_speed = s->desc.impact_speed;
  g.cutter = s->any_cutter;
  g.wait_ns = s->d.wait_ns;
  g.recolour = s->d.recolour;
  return g;
}

// One step replayed from a graph captured on first use (and again whenever
// the settings it baked in change). Two graphs alternate because the step
// swaps its double buffers. With timing on, the graph holds event-record
// nodes at the phase boundaries, pointed at this step's events before each
// replay.
tds_status step_graph(tds_scene *s, cudaEvent_t *E) {
  StepGraph &g = s->graphs[s->parity];
  const GraphKey key = graph_key(s);
  if (!g.exec || !(g.key == key)) {
    g.release();
    if (E && !s->graph_ev[0])
      for (int q = 0; q < 6; ++q) CUDA_TRY(cudaEventCreate(&s->graph_ev[q]));
    DevPtrs saved = s->d;
    uint64_t launches = 0;
    CUDA_TRY(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
    tds_status r = enqueue_step(s, E ? s->graph_ev : nullptr, launches, true);
    cudaError_t ce = cudaStreamEndCapture(s->st, &g.graph);
    s->d = saved;  // enqueue_step swapped the buffers; the replay below swaps them
    if (r != TDS_OK || ce != cudaSuccess) {
      g.release();
      if (r != TDS_OK) return r;
      return fail(TDS_ERR_CUDA, std::string("capturing the step: ") + cudaGetErrorString(ce));
    }
    if (E) {  // find the event-record nodes of the six phase boundaries
      size_t nn = 0;
      CUDA_TRY(cudaGraphGetNodes(g.graph, nullptr, &nn));
      std::vector<cudaGraphNode_t> nodes(nn);
      CUDA_TRY(cudaGraphGetNodes(g.graph, nodes.data(), &nn));
      int found = 0;
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        CUDA_TRY(cudaGraphNodeGetType(nd, &t));
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        CUDA_TRY(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        for (int q = 0; q < 6; ++q)
          if (ev == s->graph_ev[q]) { g.ev_node[q] = nd; ++found; }
      }
      if (found != 6) {
        g.release();
        return fail(TDS_ERR_CUDA, "timing graph: phase events not found");
      }
    }
    ce = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (ce != cudaSuccess) {
      g.release();
      return fail(TDS_ERR_CUDA, std::string("instantiating the step: ") + cudaGetErrorString(ce));
    }
    g.key = key;
    g.launches = launches;
  }
  if (E)
    for (int q = 0; q < 6; ++q) CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(g.exec, g.ev_node[q], E[q]));
  CUDA_TRY(cudaGraphLaunch(g.exec, s->st));
  s->launches += g.launches;
  DevPtrs &d = s->d;
  swap_state(d);  // the same swaps as the captured step
  d.targ = s->recording ? s->x.targ : nullptr;
  return TDS_OK;
}

tds_status read_particles_impl(tds_scene *s, uint32_t off, uint32_t count, float *x, float *y, float *z,
                               float *vx, float *vy, float *vz, float *wx, float *wy, float *wz) {
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  tds_launch_stage(s->d, s->L.n, s->st);
  float *outs[9] = {x, y, z, vx, vy, vz, wx, wy, wz};
  for (int q = 0; q < 9; ++q)
    if (outs[q])
      CUDA_TRY(cudaMemcpyAsync(outs[q], s->d.stage + (size_t)q * s->L.n + off, sizeof(float) * count,
                               cudaMemcpyDeviceToHost, s->st));
  return sync_and_check(s);
}

// ---- checkpoint / resume -------------------------------------------------
// What a step carries into the next: particle records in slot order, the
// warm-start memory written by the last step (buffer 0 after its swap), the
// heightfield with its pending mass and highest heights, the tool poses and
// the step count. Everything else is rebuilt by every step.
struct StateHeader {
  uint32_t magic, version, n, cap, nheights, nscenes;
  uint64_t steps;
  uint32_t have_prev, reserved;
};
constexpr uint32_t kStateMagic = 0x53534454u;  // "TDSS"
constexpr uint32_t kStateVersion = 1u;

struct StatePart {
  void *dev;
  size_t bytes;
};

std::vector<StatePart> state_parts(tds_scene *s) {
  DevPtrs &d = s->d;
  const size_t n = s->L.n, cap = s->L.cap, nh = s->L.nheights;
  return {{d.pos, 16 * n},           {d.pv, 32 * n},           {d.pid, 4 * n},
          {d.sid, 4 * n},            {d.prev_first[0], 4 * n}, {d.prev_cnt[0], 4 * n},
          {d.prev_other[0], 4 * cap}, {d.prev_l0[0], 16 * cap}, {d.prev_l1[0], 16 * cap},
          {s->x.heights, 4 * nh},    {d.hf_pend, 4 * nh},      {d.hf_top, 4 * nh}};
}

uint64_t state_bytes(tds_scene *s) {
  uint64_t b = sizeof(StateHeader) + 13 * sizeof(float) * (uint64_t)s->scenes.size();
  for (const StatePart &p : state_parts(s)) b += p.bytes;
  return b;
}

}  // namespace

// Lets other translation units of the library report through tds_last_error.
tds_status tds_set_error_message(tds_status s, const char *msg) { return fail(s, msg); }

extern "C" {

const char *tds_last_error(void) { return g_err.c_str(); }

tds_status tds_workspace_bytes(const tds_scene_desc *desc, uint64_t *bytes) {
  return workspace_bytes_impl(desc, desc ? 1u : 0u, bytes);
}

tds_status tds_batch_workspace_bytes(const tds_scene_desc *descs, uint32_t count, uint64_t *bytes) {
  return workspace_bytes_impl(descs, count, bytes);
}

tds_status tds_create_scene(const tds_scene_desc *desc, void *workspace, uint64_t workspace_bytes,
                            void *stream, tds_scene **out) {
  if (!desc) return fail(TDS_ERR_INVALID_ARG, "desc is NULL");
  return create_impl(desc, 1, workspace, workspace_bytes, stream, out);
}

tds_status tds_create_batch(const tds_scene_desc *descs, uint32_t count, void *workspace,
                            uint64_t workspace_bytes, void *stream, tds_scene **out) {
  return create_impl(descs, count, workspace, workspace_bytes, stream, out);
}

tds_status tds_set_tool_pose(tds_scene *s, const float pos[3], const float quat[4],
                             const float linvel[3], const float angvel[3]) {
  return set_pose_impl(s, 0, pos, quat, linvel, angvel);
}

tds_status tds_batch_set_tool_pose(tds_scene *s, uint32_t scene, const float pos[3], const float quat[4],
                                   const float linvel[3], const float angvel[3]) {
  return set_pose_impl(s, scene, pos, quat, linvel, angvel);
}

tds_status tds_batch_set_tool_poses(tds_scene *s, const float *poses, uint32_t count) {
  if (!s || !poses) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (count != s->scenes.size()) return fail(TDS_ERR_INVALID_ARG, "count differs from the batch size");
  for (uint32_t q = 0; q < count; ++q) {
    const float *p = poses + 13 * (size_t)q;
    tds_status r = set_pose_impl(s, q, p, p + 3, p + 7, p + 10);
    if (r != TDS_OK) return r;
  }
  return TDS_OK;
}

tds_status tds_state_bytes(tds_scene *s, uint64_t *bytes) {
  if (!s || !bytes) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  *bytes = state_bytes(s);
  return TDS_OK;
}

tds_status tds_save_state(tds_scene *s, void *buf, uint64_t bytes) {
  if (!s || !buf) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (bytes < state_bytes(s)) return fail(TDS_ERR_INVALID_ARG, "buffer smaller than tds_state_bytes()");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  tds_status r = sync_and_check(s);  // the state of the last completed step
  if (r != TDS_OK) return r;
  unsigned char *o = static_cast<unsigned char *>(buf);
  StateHeader h{kStateMagic, kStateVersion, s->L.n, s->L.cap, s->L.nheights, (uint32_t)s->scenes.size(),
                s->steps, s->have_prev ? 1u : 0u, 0u};
  std::memcpy(o, &h, sizeof h);
  o += sizeof h;
  for (const SceneHost &q : s->scenes) {
    float pose[13];
    std::memcpy(pose, q.pos, 12);
    std::memcpy(pose + 3, q.quat, 16);
    std::memcpy(pose + 7, q.vel, 12);
    std::memcpy(pose + 10, q.angvel, 12);
    std::memcpy(o, pose, sizeof pose);
    o += sizeof pose;
  }
  for (const StatePart &p : state_parts(s)) {
    CUDA_TRY(cudaMemcpyAsync(o, p.dev, p.bytes, cudaMemcpyDeviceToHost, s->st));
    o += p.bytes;
  }
  CUDA_TRY(cudaStreamSynchronize(s->st));
  return TDS_OK;
}

tds_status tds_load_state(tds_scene *s, const void *buf, uint64_t bytes) {
  if (!s || !buf) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (bytes < sizeof(StateHeader)) return fail(TDS_ERR_INVALID_ARG, "buffer too small for a state");
  StateHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (h.magic != kStateMagic || h.version != kStateVersion)
    return fail(TDS_ERR_INVALID_ARG, "not a saved scene state (or another version)");
  if (h.n != s->L.n || h.cap != s->L.cap || h.nheights != s->L.nheights || h.nscenes != s->scenes.size())
    return fail(TDS_ERR_INVALID_ARG, "state saved from a scene of another layout (particles, capacity, "
                                     "heightfield or scene count)");
  if (bytes < state_bytes(s)) return fail(TDS_ERR_INVALID_ARG, "buffer shorter than the state");
  CUDA_TRY(cudaStreamSynchronize(s->st));
  const unsigned char *o = static_cast<const unsigned char *>(buf) + sizeof h;
  for (uint32_t q = 0; q < h.nscenes; ++q) {
    float pose[13];
    std::memcpy(pose, o, sizeof pose);
    o += sizeof pose;
    tds_status r = set_pose_impl(s, q, pose, pose + 3, pose + 7, pose + 10);
    if (r != TDS_OK) return r;
  }
  for (const StatePart &p : state_parts(s)) {
    CUDA_TRY(cudaMemcpyAsync(p.dev, o, p.bytes, cudaMemcpyHostToDevice, s->st));
    o += p.bytes;
  }
  const int32_t zero = 0;
  const uint32_t clean = (uint32_t)h.steps;
  CUDA_TRY(cudaMemcpyAsync(s->d.err, &zero, sizeof zero, cudaMemcpyHostToDevice, s->st));
  CUDA_TRY(cudaMemcpyAsync(s->d.ctr + CTR_CLEAN, &clean, sizeof clean, cudaMemcpyHostToDevice, s->st));
  CUDA_TRY(cudaStreamSynchronize(s->st));
  s->steps = h.steps;
  s->have_prev = h.have_prev != 0;
  s->latched = TDS_OK;
  return TDS_OK;
}

tds_status tds_set_solver(tds_scene *s, uint32_t max_iters, float tol, uint32_t residual_every) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  if (max_iters == 0 || !(tol >= 0.f)) return fail(TDS_ERR_INVALID_ARG, "max_iters >= 1 and tol >= 0 required");
  s->desc.max_iters = max_iters;
  s->desc.tol = tol;
  s->desc.residual_every = residual_every;  // 0: adaptive checks
  return TDS_OK;
}

tds_status tds_set_impact(tds_scene *s, float restitution, float impact_speed, uint32_t impact_iters) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  if (!(restitution >= 0.f && restitution <= 1.f) || !(impact_speed >= 0.f) || !std::isfinite(impact_speed))
    return fail(TDS_ERR_INVALID_ARG, "restitution must be in [0, 1] and impact_speed >= 0");
  s->desc.restitution = restitution;
  s->desc.impact_speed = impact_speed;
  s->desc.impact_iters = impact_iters;
  return TDS_OK;
}

tds_status tds_set_recolour_period(tds_scene *s, uint32_t period) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  if (period == 0) return fail(TDS_ERR_INVALID_ARG, "period must be >= 1");
  s->d.recolour = period;
  return TDS_OK;
}

tds_status tds_set_warm_start(tds_scene *s, int32_t mode) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  if (mode != TDS_WARM_COLD && mode != TDS_WARM_PREV && mode != TDS_WARM_LEARNED)
    return fail(TDS_ERR_INVALID_ARG, "unknown warm start");
  s->desc.warm_start = mode;
  return TDS_OK;
}

tds_status tds_get_launch_config(tds_scene *s, tds_launch_config *out) {
  if (!s || !out) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  out->pgs_blocks = s->pgs_blocks;
  out->pgs_sync = s->pgs_sync;
  out->colour_blocks = s->colour_blocks;
  out->max_pgs_blocks = std::min(s->max_pgs_blocks, s->sms * tds_pgs_occupancy(s->pgs_shape));
  out->max_colour_blocks = s->max_colour_blocks;
  tds_pgs_shape(s->pgs_shape, &out->pgs_threads, &out->pgs_per_thread);
  out->wait_limit_us = (int32_t)(s->d.wait_ns / 1000ull);
  return TDS_OK;
}

tds_status tds_set_launch_config(tds_scene *s, const tds_launch_config *cfg) {
  if (!s || !cfg) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (cfg->pgs_blocks < 0 || cfg->colour_blocks < 0 ||
      cfg->colour_blocks > s->max_colour_blocks || (cfg->pgs_sync != 0 && cfg->pgs_sync != 1) ||
      cfg->wait_limit_us < 0)
    return fail(TDS_ERR_INVALID_ARG,
                "pgs_blocks and colour_blocks must be in [0, max] (0 keeps the value), pgs_sync 0 or 1, "
                "wait_limit_us >= 0");
  int shape = s->pgs_shape;
  if (cfg->pgs_threads || cfg->pgs_per_thread) {
    shape = -1;
    for (int i = 0; i < tds_pgs_shapes(); ++i) {
      int t = 0, per = 0;
      tds_pgs_shape(i, &t, &per);
      if (t == cfg->pgs_threads && per == cfg->pgs_per_thread) shape = i;
    }
    if (shape < 0) {
      std::string known;
      for (int i = 0; i < tds_pgs_shapes(); ++i) {
        int t = 0, per = 0;
        tds_pgs_shape(i, &t, &per);
        known += (i ? ", " : "") + std::to_string(t) + "x" + std::to_string(per);
      }
      return fail(TDS_ERR_INVALID_ARG, "pgs_threads x pgs_per_thread must be a compiled shape (" + known +
                                           ") or both 0");
    }
  }
  // the solver CTAs must all be co-resident: at most the SMs times the
  // chosen shape's CTAs per SM
  const int max_blocks = std::min(64 * s->sms, s->sms * tds_pgs_occupancy(shape));
  if (cfg->pgs_blocks > max_blocks)
    return fail(TDS_ERR_INVALID_ARG, "pgs_blocks exceeds the co-resident CTAs of that solver shape (" +
                                         std::to_string(max_blocks) + ")");
  if (cfg->pgs_blocks) s->pgs_blocks = cfg->pgs_blocks;
  else if (s->pgs_blocks > max_blocks) s->pgs_blocks = max_blocks;
  if (cfg->colour_blocks) s->colour_blocks = cfg->colour_blocks;
  if (cfg->wait_limit_us) s->d.wait_ns = 1000ull * (unsigned long long)cfg->wait_limit_us;
  s->pgs_sync = cfg->pgs_sync;
  s->pgs_shape = shape;
  return TDS_OK;
}

tds_status tds_set_graph(tds_scene *s, int32_t enable) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  if (enable && (s->st == nullptr || s->st == cudaStreamLegacy || s->st == cudaStreamPerThread))
    return fail(TDS_ERR_INVALID_ARG, "graph replay needs a created (non-default) stream");
  s->graph = enable != 0;
  return TDS_OK;
}

tds_status tds_step(tds_scene *s, uint32_t nsteps) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  if (s->desc.warm_start == TDS_WARM_LEARNED && !s->have_weights)
    return fail(TDS_ERR_STATE, "TDS_WARM_LEARNED needs tds_set_mlp_weights first");
  for (uint32_t it = 0; it < nsteps; ++it) {
    if (s->geo_dirty) {  // tool poses changed: new world boxes and tool motion
      CUDA_TRY(cudaMemcpyAsync(s->x.boxes, s->host_boxes.data(), sizeof(BoxF) * s->host_boxes.size(),
                               cudaMemcpyHostToDevice, s->st));
      CUDA_TRY(cudaMemcpyAsync(s->x.geo, s->L.geo.data(), sizeof(SceneGeo) * s->L.geo.size(),
                               cudaMemcpyHostToDevice, s->st));
      s->geo_dirty = false;
    }
    cudaEvent_t *E = nullptr;
    if (s->timing) {
      while (s->ev.size() < s->ev_used + 6) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        s->ev.push_back(e);
      }
      E = s->ev.data() + s->ev_used;
      s->ev_used += 6;
    }
    tds_status r = s->graph ? step_graph(s, E) : enqueue_step(s, E, s->launches);
    if (r != TDS_OK) return r;
    s->parity ^= 1u;
    s->have_prev = true;
    s->steps++;
  }
  CUDA_TRY(cudaGetLastError());
  return TDS_OK;
}

tds_status tds_synchronize(tds_scene *s) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  return sync_and_check(s);
}

tds_status tds_read_particles(tds_scene *s, float *x, float *y, float *z, float *vx, float *vy,
                              float *vz, float *wx, float *wy, float *wz, uint32_t n) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  if (n != s->L.n) return fail(TDS_ERR_INVALID_ARG, "n differs from the scene's particle count");
  return read_particles_impl(s, 0, n, x, y, z, vx, vy, vz, wx, wy, wz);
}

tds_status tds_set_cutter(tds_scene *s, uint32_t scene, const tds_cutter *c) {
  if (!s || !c) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (scene >= s->scenes.size()) return fail(TDS_ERR_INVALID_ARG, "scene index out of range");
  const SceneGeo &G = s->L.geo[scene];
  if (c->length > 0.f) {
    if (G.hf_nx <= 0) return fail(TDS_ERR_INVALID_ARG, "a cutter needs the scene's heightfield");
    const float rmax = s->L.rmax;
    if (!(c->spawn_radius > 0.f) || c->spawn_radius > rmax || 2.f * c->spawn_radius > G.hf_cell)
      return fail(TDS_ERR_INVALID_ARG,
                  "spawn_radius must be in (0, largest radius at creation] and at most half the heightfield cell");
    if (!(c->bank_density > 0.f) || !(c->phi >= 0.f && c->phi < 1.5707963f))
      return fail(TDS_ERR_INVALID_ARG, "bank_density > 0 and 0 <= phi < pi/2 required");
    const double du = std::sqrt((double)c->dir[0] * c->dir[0] + (double)c->dir[1] * c->dir[1] +
                                (double)c->dir[2] * c->dir[2]);
    const double dn = std::sqrt((double)c->normal[0] * c->normal[0] + (double)c->normal[1] * c->normal[1] +
                                (double)c->normal[2] * c->normal[2]);
    if (!(du > 1e-9) || !(dn > 1e-9) || !std::isfinite(c->length))
      return fail(TDS_ERR_INVALID_ARG, "edge direction and blade normal must be non-zero");
  }
  SceneHost &h = s->scenes[scene];
  h.cutter = *c;
  h.has_cutter = c->length > 0.f;
  compose_boxes(s, scene);
  s->any_cutter = false;
  for (const SceneHost &q : s->scenes) s->any_cutter |= q.has_cutter;
  return TDS_OK;
}

tds_status tds_read_heightfield(tds_scene *s, uint32_t scene, float *heights, float *pending, uint32_t count) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  if (scene >= s->scenes.size()) return fail(TDS_ERR_INVALID_ARG, "scene index out of range");
  const SceneGeo &G = s->L.geo[scene];
  const uint32_t nodes = G.hf_nx > 0 ? (uint32_t)((G.hf_nx + 1) * (G.hf_ny + 1)) : 0u;
  if (count != nodes) return fail(TDS_ERR_INVALID_ARG, "count differs from the scene's heightfield nodes");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  if (nodes && heights)
    CUDA_TRY(cudaMemcpyAsync(heights, s->x.heights + G.hf_off, sizeof(float) * nodes, cudaMemcpyDeviceToHost,
                             s->st));
  if (nodes && pending)
    CUDA_TRY(cudaMemcpyAsync(pending, s->d.hf_pend + G.hf_off, sizeof(float) * nodes, cudaMemcpyDeviceToHost,
                             s->st));
  return sync_and_check(s);
}

tds_status tds_read_radii(tds_scene *s, float *r, uint32_t n) {
  if (!s || !r) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (n != s->L.n) return fail(TDS_ERR_INVALID_ARG, "n differs from the particle count");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  tds_launch_stage(s->d, s->L.n, s->st);
  CUDA_TRY(cudaMemcpyAsync(r, s->d.stage + (size_t)9 * s->L.n, sizeof(float) * n, cudaMemcpyDeviceToHost, s->st));
  return sync_and_check(s);
}

tds_status tds_batch_read_particles(tds_scene *s, uint32_t scene, float *x, float *y, float *z, float *vx,
                                    float *vy, float *vz, float *wx, float *wy, float *wz, uint32_t n) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  if (scene >= s->scenes.size()) return fail(TDS_ERR_INVALID_ARG, "scene index out of range");
  if (n != s->scenes[scene].n) return fail(TDS_ERR_INVALID_ARG, "n differs from that scene's particle count");
  return read_particles_impl(s, s->scenes[scene].off, n, x, y, z, vx, vy, vz, wx, wy, wz);
}

tds_status tds_read_tool_force(tds_scene *s, float force[3], float torque[3]) {
  if (!s || !force || !torque) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  float buf[6];
  CUDA_TRY(cudaMemcpyAsync(buf, s->d.tool_out, sizeof(buf), cudaMemcpyDeviceToHost, s->st));
  tds_status r = sync_and_check(s);
  if (r != TDS_OK) return r;
  for (int i = 0; i < 3; ++i) { force[i] = buf[i]; torque[i] = buf[3 + i]; }
  return TDS_OK;
}

tds_status tds_batch_read_tool_forces(tds_scene *s, float *force_torque, uint32_t count) {
  if (!s || !force_torque) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (count != s->scenes.size()) return fail(TDS_ERR_INVALID_ARG, "count differs from the batch size");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  CUDA_TRY(cudaMemcpyAsync(force_torque, s->d.tool_out, sizeof(float) * 6 * count, cudaMemcpyDeviceToHost, s->st));
  return sync_and_check(s);
}

tds_status tds_batch_read_solve(tds_scene *s, float *residual, uint32_t *sweeps, uint32_t count) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (count != s->scenes.size()) return fail(TDS_ERR_INVALID_ARG, "count differs from the batch size");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  if (residual)
    CUDA_TRY(cudaMemcpyAsync(residual, s->d.scene_res, sizeof(float) * count, cudaMemcpyDeviceToHost, s->st));
  if (sweeps)
    CUDA_TRY(cudaMemcpyAsync(sweeps, s->d.scene_iters, sizeof(uint32_t) * count, cudaMemcpyDeviceToHost, s->st));
  return sync_and_check(s);
}

tds_status tds_get_stats(tds_scene *s, tds_step_stats *out) {
  if (!s || !out) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  uint32_t ctr[CTR_COUNT];
  unsigned long long acc[ACC_COUNT];
  float fs[FS_COUNT];
  std::vector<uint32_t> bs(TDS_NBUCKETS + 1), be(TDS_NBUCKETS);
  CUDA_TRY(cudaMemcpyAsync(ctr, s->d.ctr, sizeof(ctr), cudaMemcpyDeviceToHost, s->st));
  CUDA_TRY(cudaMemcpyAsync(fs, s->d.fscal, sizeof(fs), cudaMemcpyDeviceToHost, s->st));
  CUDA_TRY(cudaMemcpyAsync(acc, s->d.acc, sizeof(acc), cudaMemcpyDeviceToHost, s->st));
  CUDA_TRY(cudaMemsetAsync(s->d.acc, 0, sizeof(acc), s->st));
  CUDA_TRY(cudaMemcpyAsync(bs.data(), s->d.bstart, sizeof(uint32_t) * bs.size(), cudaMemcpyDeviceToHost, s->st));
  CUDA_TRY(cudaMemcpyAsync(be.data(), s->d.bend, sizeof(uint32_t) * be.size(), cudaMemcpyDeviceToHost, s->st));
  tds_status r = sync_and_check(s);
  if (r != TDS_OK) return r;
  std::memset(out, 0, sizeof(*out));
  out->n_contacts = ctr[CTR_NC];
  uint32_t nst = 0;
  for (int c = 0; c < TDS_MAX_COLOURS; ++c) nst += be[2 * c + 1] - bs[2 * c + 1];
  out->n_static = nst;
  out->n_pp = ctr[CTR_NC] - nst;
  out->n_colours = ctr[CTR_NCOL];
  out->colour_rounds = ctr[CTR_ROUNDS];
  out->impacts = s->desc.impact_iters ? ctr[CTR_IMPACTS] : 0;
  out->spawned = s->any_cutter ? ctr[CTR_SPAWN] : 0;
  out->iterations = ctr[CTR_ITERS];
  out->residual = fs[FS_RESID];
  out->steps = s->steps;
  out->kernel_launches = s->launches;
  out->sweep_contacts_pp = acc[ACC_SWEEP_PP];
  out->sweep_contacts_static = acc[ACC_SWEEP_ST];
  out->sum_contacts = acc[ACC_CONTACTS];
  out->solved_steps = acc[ACC_STEPS];
  out->timed_steps = (uint32_t)(s->ev_used / 6);
  for (size_t b = 0; b + 6 <= s->ev_used; b += 6)
    for (int q = 0; q < 5; ++q) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, s->ev[b + q], s->ev[b + q + 1]));
      out->phase_ms[q] += ms;
    }
  s->ev_used = 0;
  return TDS_OK;
}

tds_status tds_set_timing(tds_scene *s, int32_t enable) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  s->timing = enable != 0;
  s->ev_used = 0;
  return TDS_OK;
}

tds_status tds_read_contacts(tds_scene *s, uint64_t *keys, float *lam, uint32_t *colour,
                             uint32_t cap, uint32_t *count) {
  if (!s || !count) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  uint32_t nc = 0;
  CUDA_TRY(cudaMemcpyAsync(&nc, s->d.ctr + CTR_NC, sizeof(nc), cudaMemcpyDeviceToHost, s->st));
  tds_status r = sync_and_check(s);
  if (r != TDS_OK) return r;
  *count = nc;
  uint32_t m = nc < cap ? nc : cap;
  if (m == 0 || !s->have_prev) return TDS_OK;
  std::vector<float4> l0(m), l1(m);
  if (keys) CUDA_TRY(cudaMemcpyAsync(keys, s->d.c_key, sizeof(uint64_t) * m, cudaMemcpyDeviceToHost, s->st));
  if (colour) {
    std::vector<uint8_t> col(m);
    CUDA_TRY(cudaMemcpyAsync(col.data(), s->d.colour, m, cudaMemcpyDeviceToHost, s->st));
    CUDA_TRY(cudaStreamSynchronize(s->st));
    for (uint32_t i = 0; i < m; ++i) colour[i] = col[i];
  }
  if (lam) {
    CUDA_TRY(cudaMemcpyAsync(l0.data(), s->d.prev_l0[0], sizeof(float4) * m, cudaMemcpyDeviceToHost, s->st));
    CUDA_TRY(cudaMemcpyAsync(l1.data(), s->d.prev_l1[0], sizeof(float4) * m, cudaMemcpyDeviceToHost, s->st));
  }
  CUDA_TRY(cudaStreamSynchronize(s->st));
  if (lam)
    for (uint32_t i = 0; i < m; ++i) {
      float *o = lam + 7 * (size_t)i;
      o[0] = l0[i].x; o[1] = l0[i].y; o[2] = l0[i].z; o[3] = l0[i].w;
      o[4] = l1[i].x; o[5] = l1[i].y; o[6] = l1[i].z;
    }
  return TDS_OK;
}

tds_status tds_aggregate_bodies(tds_scene *s, const tds_zone *zones, uint32_t count, tds_aggregate *out) {
  if (!s || (count && (!zones || !out))) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (count > TDS_MAX_ZONES) return fail(TDS_ERR_INVALID_ARG, "more than TDS_MAX_ZONES zones");
  for (uint32_t z = 0; z < count; ++z) {
    if (zones[z].scene >= s->scenes.size()) return fail(TDS_ERR_INVALID_ARG, "zone scene out of range");
    if (zones[z].n_planes < 1 || zones[z].n_planes > TDS_ZONE_MAX_PLANES)
      return fail(TDS_ERR_INVALID_ARG, "zone needs 1..TDS_ZONE_MAX_PLANES planes");
    for (uint32_t k = 0; k < zones[z].n_planes; ++k)
      for (int q = 0; q < 4; ++q)
        if (!std::isfinite(zones[z].planes[k][q])) return fail(TDS_ERR_INVALID_ARG, "non-finite zone plane");
  }
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  if (count == 0) return TDS_OK;
  CUDA_TRY(cudaMemcpyAsync(s->x.zones, zones, sizeof(tds_zone) * count, cudaMemcpyHostToDevice, s->st));
  s->launches += tds_launch_aggregate(s->d, s->L.n, s->x.zones, count, s->x.zone_id, s->x.agg_sums,
                                      s->x.agg_out, s->st);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(out, s->x.agg_out, sizeof(tds_aggregate) * count, cudaMemcpyDeviceToHost, s->st));
  return sync_and_check(s);
}

tds_status tds_coarse_grain(tds_scene *s, const tds_grid *grid, int32_t kernel, float R, float *rho, float *p,
                            float *u) {
  if (!s || !rho || !p || !u) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (!tds_grid_valid(grid)) return fail(TDS_ERR_INVALID_ARG, "invalid grid");
  if (grid->scene >= s->scenes.size()) return fail(TDS_ERR_INVALID_ARG, "grid scene out of range");
  if (kernel != 0 && kernel != 1) return fail(TDS_ERR_INVALID_ARG, "kernel must be 0 (voxel) or 1 (Gaussian)");
  if (kernel == 1 && !(R > 0.0f && R <= 16.0f * grid->l0))
    return fail(TDS_ERR_INVALID_ARG, "Gaussian smoothing length must be in (0, 16 l0]");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  s->launches += tds_launch_coarse_grain(s->d, s->L.n, *grid, kernel, R, rho, p, u, s->st);
  CUDA_TRY(cudaGetLastError());
  return TDS_OK;
}

tds_status tds_set_mlp_weights(tds_scene *s, const float *params, uint32_t count) {
  if (!s || !params) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if ((int)count != tds_mlp_params()) return fail(TDS_ERR_INVALID_ARG, "count must be tds_mlp_param_count()");
  CUDA_TRY(cudaMemcpyAsync(s->x.params, params, sizeof(float) * count, cudaMemcpyHostToDevice, s->st));
  tds_mlp_pack(s->x.params, s->x.packed, s->st);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s->st));
  s->have_weights = true;
  return TDS_OK;
}

tds_status tds_set_recording(tds_scene *s, int32_t enable) {
  if (!s) return fail(TDS_ERR_INVALID_ARG, "scene is NULL");
  s->recording = enable != 0;
  return TDS_OK;
}

tds_status tds_read_training_samples(tds_scene *s, float *feat, float *targ, uint64_t *keys,
                                     uint32_t cap, uint32_t *count) {
  if (!s || !count) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  tds_status ls = check_latched(s);
  if (ls != TDS_OK) return ls;
  if (!s->recording) return fail(TDS_ERR_STATE, "recording is off (tds_set_recording)");
  uint32_t nc = 0;
  CUDA_TRY(cudaMemcpyAsync(&nc, s->d.ctr + CTR_NC, sizeof(nc), cudaMemcpyDeviceToHost, s->st));
  tds_status r = sync_and_check(s);
  if (r != TDS_OK) return r;
  *count = nc;
  uint32_t m = nc < cap ? nc : cap;
  if (m == 0 || s->steps == 0) return TDS_OK;
  if (feat) CUDA_TRY(cudaMemcpyAsync(feat, s->d.feat, sizeof(float) * 10 * m, cudaMemcpyDeviceToHost, s->st));
  if (targ) CUDA_TRY(cudaMemcpyAsync(targ, s->x.targ, sizeof(float) * 3 * m, cudaMemcpyDeviceToHost, s->st));
  if (keys) CUDA_TRY(cudaMemcpyAsync(keys, s->d.c_key, sizeof(uint64_t) * m, cudaMemcpyDeviceToHost, s->st));
  CUDA_TRY(cudaStreamSynchronize(s->st));
  return TDS_OK;
}

uint32_t tds_mlp_param_count(void) { return (uint32_t)tds_mlp_params(); }

tds_status tds_mlp_workspace_bytes(uint64_t *bytes) {
  if (!bytes) return fail(TDS_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = tds_mlp_packed_bytes();
  return TDS_OK;
}

tds_status tds_mlp_forward(const float *params, const float *X, uint32_t m, float *Y, void *workspace,
                           void *stream) {
  if (!params || !X || !Y || !workspace) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  tds_mlp_pack(params, workspace, st);
  if (m) tds_mlp_forward_launch(workspace, X, m, Y, st);
  CUDA_TRY(cudaGetLastError());
  return TDS_OK;
}

tds_status tds_mlp_loss_grad(const float *params, const float *X, const float *T, uint32_t m, float *grad,
                             float *loss, void *workspace, void *stream) {
  if (!params || !X || !T || !grad || !loss || !workspace) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (m == 0) return fail(TDS_ERR_INVALID_ARG, "m must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(cudaMemsetAsync(grad, 0, sizeof(float) * tds_mlp_params(), st));
  CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
  tds_mlp_pack(params, workspace, st);
  CUDA_TRY(tds_mlp_loss_grad_launch(workspace, X, T, m, grad, loss, st));
  return TDS_OK;
}

tds_status tds_mlp_adam_step(float *params, float *grad, float *mom, float *vel, uint32_t step, float lr,
                             void *stream) {
  if (!params || !grad || !mom || !vel) return fail(TDS_ERR_INVALID_ARG, "NULL argument");
  if (step == 0 || !(lr > 0.f)) return fail(TDS_ERR_INVALID_ARG, "step >= 1 and lr > 0 required");
  tds_mlp_adam_launch(params, grad, mom, vel, step, lr, (cudaStream_t)stream);
  CUDA_TRY(cudaGetLastError());
  return TDS_OK;
}

void tds_destroy_scene(tds_scene *s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  else cudaDeviceSynchronize();
  for (StepGraph &g : s->graphs) g.release();
  for (cudaEvent_t e : s->graph_ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
  if (s->owns && s->mem) cudaFree(s->mem);
  delete s;
}

}  // extern "C"
