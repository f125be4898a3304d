// tds_cut.cu -- the active zone of a cutting edge turning terrain into
// particles (section "Mesoscale model", Eq. failure_plane): after the step's
// position update, heightfield nodes inside the wedge are lowered onto the
// failure plane, the removed mass becomes pending at the node, and a node cut
// this step places particles in its liberated column where no particle sits,
// taking dormant slots (radius 0) in id order. The cut runs over all nodes
// first; then two passes (count, write) make the same placement decisions
// from the same inputs, and scans give each node its first new particle and
// each scene its dormant ids.
#include "tds_internal.cuh"

namespace {

constexpr int kMaxPerNode = 64;

__device__ __forceinline__ void node_xy(const SceneGeo &G, uint32_t local, float &x, float &y) {
  const uint32_t i = local % (uint32_t)(G.hf_nx + 1), j = local / (uint32_t)(G.hf_nx + 1);
  x = __fadd_rn(G.hf_x0, __fmul_rn((float)i, G.hf_cell));
  y = __fadd_rn(G.hf_y0, __fmul_rn((float)j, G.hf_cell));
}

// Height zf of the failure plane above (x, y), and whether that point lies
// within the edge's length and at least rs ahead of the blade.
__device__ __forceinline__ bool in_wedge(const SceneGeo &G, float x, float y, float &zf) {
  const float dx = __fsub_rn(x, G.e0[0]), dy = __fsub_rn(y, G.e0[1]);
  zf = __fsub_rn(G.e0[2], __fdiv_rn(__fadd_rn(__fmul_rn(G.nf[0], dx), __fmul_rn(G.nf[1], dy)), G.nf[2]));
  const float dz = __fsub_rn(zf, G.e0[2]);
  const float su = __fadd_rn(__fadd_rn(__fmul_rn(G.u[0], dx), __fmul_rn(G.u[1], dy)), __fmul_rn(G.u[2], dz));
  const float ahead =
      __fadd_rn(__fadd_rn(__fmul_rn(G.ns[0], dx), __fmul_rn(G.ns[1], dy)), __fmul_rn(G.ns[2], dz));
  return su >= 0.0f && su <= G.cut_len && ahead >= G.rs;
}

// No active particle of the scene overlaps a sphere of radius rs at c (FP32
// test (dx^2 + dy^2) + dz^2 < (rs + r)^2 means overlap). The search covers the
// cells within two of c's cell in this step's broadphase; the spawn radius is
// at most the largest radius, so two cells cover every possible overlap even
// after the step's motion.
__device__ bool free_at(const DevPtrs &d, const StepConsts &k, const SceneGeo &G, uint32_t scene, float cx_,
                        float cy_, float cz_) {
  int cx, cy, cz;
  (void)cell_index(k, G, scene, make_float4(cx_, cy_, cz_, G.rs), cx, cy, cz);
  const uint32_t block = scene * (uint32_t)k.gnx * (uint32_t)k.gny * (uint32_t)k.gnz;
  const int z0 = max(cz - 2, 0), z1 = min(cz + 2, k.gnz - 1);
  for (int x = max(cx - 2, 0); x <= min(cx + 2, k.gnx - 1); ++x)
    for (int y = max(cy - 2, 0); y <= min(cy + 2, k.gny - 1); ++y) {
      const uint32_t row = block + ((uint32_t)x * (uint32_t)k.gny + (uint32_t)y) * (uint32_t)k.gnz;
      const uint32_t s = d.cell_start[row + z0], e = d.cell_start[row + z1 + 1];
      for (uint32_t q = s; q < e; ++q) {
        const float4 P = d.pos[q];
        if (P.w == 0.0f) continue;
        const float dx = __fsub_rn(cx_, P.x), dy = __fsub_rn(cy_, P.y), dz = __fsub_rn(cz_, P.z);
        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        const float rr = __fadd_rn(G.rs, P.w);
        if (d2 < __fmul_rn(rr, rr)) return false;
      }
    }
  return true;
}

// Largest sqrt((cell^2 + A^2) + B^2) over the heightfield triangles around a
// node, A and B a triangle's height steps along its legs (lower triangle of
// cell (a, b): corners (a, b), (a+1, b), (a, b+1); upper: (a+1, b+1),
// (a, b+1), (a+1, b)). Every such plane passes through the node, so a point
// z above the node lies cell (z - zf) / den from the nearest of them.
__device__ float node_den(const SceneGeo &G, const float *heights, uint32_t local) {
  const int w = G.hf_nx + 1, i = (int)(local % (uint32_t)w), j = (int)(local / (uint32_t)w);
  const float *H = heights + G.hf_off;
  const float c2 = __fmul_rn(G.hf_cell, G.hf_cell);
  constexpr int kTri[6][3] = {{0, 0, 0}, {-1, 0, 0}, {-1, 0, 1}, {0, -1, 0}, {0, -1, 1}, {-1, -1, 1}};
  float dmax = G.hf_cell;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int a = i + kTri[t][0], b = j + kTri[t][1];
    if (a < 0 || b < 0 || a >= G.hf_nx || b >= G.hf_ny) continue;
    float hb, A, B;
    if (!kTri[t][2]) {
      hb = H[b * w + a];
      A = __fsub_rn(H[b * w + a + 1], hb);
      B = __fsub_rn(H[(b + 1) * w + a], hb);
    } else {
      hb = H[(b + 1) * w + a + 1];
      A = __fsub_rn(H[(b + 1) * w + a], hb);
      B = __fsub_rn(H[b * w + a + 1], hb);
    }
    dmax = fmaxf(dmax, __fsqrt_rn(__fadd_rn(__fadd_rn(c2, __fmul_rn(A, A)), __fmul_rn(B, B))));
  }
  return dmax;
}

// First-fit placement up the liberated column [zf, top]: calls take(z) for
// each accepted position while the pending mass pays; returns the count. A
// position is accepted when it clears the planes of the terrain triangles
// around the node (after this step's cut) by rs and no active particle
// overlaps it.
template <class F>
__device__ uint32_t place(const DevPtrs &d, const StepConsts &k, const SceneGeo &G, uint32_t scene, uint32_t local,
                          float zf, float top, float pend, F &&take) {
  float x, y;
  node_xy(G, local, x, y);
  const float den = node_den(G, k.heights, local);
  const float two_rs = __fmul_rn(2.0f, G.rs);
  uint32_t n = 0;
  float rem = pend;
  for (int j = 0; j < kMaxPerNode; ++j) {
    const float z = __fadd_rn(zf, __fadd_rn(G.rs, __fmul_rn(two_rs, (float)j)));
    if (__fadd_rn(z, G.rs) > top || rem < G.ms) break;
    if (__fdiv_rn(__fmul_rn(G.hf_cell, __fsub_rn(z, zf)), den) < G.rs) continue;
    if (!free_at(d, k, G, scene, x, y, z)) continue;
    take(n, z);
    ++n;
    rem = __fsub_rn(rem, G.ms);
  }
  return n;
}

// The cut: nodes in the wedge lowered onto the failure plane, the removed
// mass added to their pending mass; hf_cnt marks the nodes cut this step.
__global__ void k_cut(DevPtrs d, StepConsts k, float *heights, uint32_t nh) {
  if (step_failed(d)) return;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nh; q += gridDim.x * blockDim.x) {
    const uint32_t scene = d.hf_scene[q];
    const SceneGeo &G = k.geo[scene];
    uint32_t cut = 0;
    float x, y, zf;
    if (G.cut_on) {
      node_xy(G, q - G.hf_off, x, y);
      const float h = heights[q];
      if (in_wedge(G, x, y, zf) && h > zf) {
        const float dh = __fsub_rn(h, zf);
        heights[q] = zf;
        d.hf_pend[q] =
            __fadd_rn(d.hf_pend[q], __fmul_rn(__fmul_rn(__fmul_rn(G.rho_b, dh), G.hf_cell), G.hf_cell));
        cut = 1;
      }
    }
    d.hf_cnt[q] = cut;
  }
}

// Particles each node cut this step can place (all cuts done: the terrain
// test sees the final heights).
__global__ void k_cut_count(DevPtrs d, StepConsts k, const float *heights, uint32_t nh) {
  if (step_failed(d)) return;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nh; q += gridDim.x * blockDim.x) {
    if (!d.hf_cnt[q]) continue;
    const uint32_t scene = d.hf_scene[q];
    const SceneGeo &G = k.geo[scene];
    d.hf_cnt[q] = place(d, k, G, scene, q - G.hf_off, heights[q], d.hf_top[q], d.hf_pend[q], [](uint32_t, float) {});
  }
}

// Dormant slots: their ids flagged (then scanned into ranks), listed by rank,
// and each id's slot.
__global__ void k_dorm_flags(DevPtrs d, uint32_t n) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
    d.dorm_rank[d.pid[s]] = d.pos[s].w == 0.0f ? 1u : 0u;
}
__global__ void k_dorm_list(DevPtrs d, uint32_t n) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    if (d.pos[s].w != 0.0f) continue;
    const uint32_t pid = d.pid[s];
    d.dorm_list[d.dorm_rank[pid]] = pid;
    d.slot_of_pid[pid] = s;
  }
}

__global__ void k_cut_write(DevPtrs d, StepConsts k, const float *heights, uint32_t nh) {
  if (step_failed(d)) return;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nh; q += gridDim.x * blockDim.x) {
    const uint32_t cnt = d.hf_cnt[q];
    if (cnt == 0) continue;
    const uint32_t scene = d.hf_scene[q];
    const SceneGeo &G = k.geo[scene];
    float x, y;
    node_xy(G, q - G.hf_off, x, y);
    const uint32_t r0 = d.hf_rank[q] - d.hf_rank[G.hf_off];
    const uint32_t dbase = d.dorm_rank[G.pid0], davail = d.dorm_rank[G.pid0 + G.npart] - dbase;
    uint32_t taken = 0;
    const float pend = d.hf_pend[q];
    place(d, k, G, scene, q - G.hf_off, heights[q], d.hf_top[q], pend, [&](uint32_t a, float z) {
      const uint32_t r = r0 + a;
      if (r >= davail) return;
      const uint32_t pid = d.dorm_list[dbase + r], s = d.slot_of_pid[pid];
      d.pos[s] = make_float4(x, y, z, G.rs);
      d.pv[2 * (size_t)s] = make_float4(0.f, 0.f, 0.f, G.inv_m);
      d.pv[2 * (size_t)s + 1] = make_float4(0.f, 0.f, 0.f, G.inv_I);
      ++taken;
    });
    d.hf_pend[q] = __fsub_rn(pend, __fmul_rn((float)taken, G.ms));
    if (taken) atomicAdd(d.ctr + CTR_SPAWN, taken);
  }
}

unsigned blocks_for(uint32_t n) {
  unsigned b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 8) b = 152 * 8;
  return b;
}

}  // namespace

int tds_launch_cut(const DevPtrs &d, const StepConsts &k, float *heights, uint32_t nh, cudaStream_t st) {
  cudaMemsetAsync(d.ctr + CTR_SPAWN, 0, sizeof(uint32_t), st);
  k_dorm_flags<<<blocks_for(k.n), 256, 0, st>>>(d, k.n);
  tds_scan_exclusive(d.dorm_rank, d.dorm_rank, k.n, d.scan_tmp, st);
  k_dorm_list<<<blocks_for(k.n), 256, 0, st>>>(d, k.n);
  k_cut<<<blocks_for(nh), 256, 0, st>>>(d, k, heights, nh);
  k_cut_count<<<blocks_for(nh), 256, 0, st>>>(d, k, heights, nh);
  tds_scan_exclusive(d.hf_cnt, d.hf_rank, nh, d.scan_tmp, st);
  k_cut_write<<<blocks_for(nh), 256, 0, st>>>(d, k, heights, nh);
  return 11;
}
