// tds_internal.cuh -- device-side types and helpers shared by the kernels of
// libtds (the GB300 particle step). Nothing here is visible through the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tds.h"

#define TDS_STATIC 0x80000000u
#define TDS_NO_COLOUR 0xFFu
#define TDS_MAX_COLOURS 128
#define TDS_NBUCKETS (2 * TDS_MAX_COLOURS)  // (colour, static?) buckets
#define TDS_TILE 2048                       // contacts per bucketing tile
#define TDS_ORDER_PAD (4 * TDS_NBUCKETS + 16) // padding slots of the colour order
#define TDS_RES_CHUNK 256u                  // contacts per residual chunk (at most)
#define TDS_BARRIER_NS 2000000000ull        // default limit of a wait on other CTAs (2 s); also the
                                            // fixed limit of a CTA's wait for its own bulk copies

// Error codes latched on the device (the tds_status values).
#define DEV_ERR_CAPACITY (-4)
#define DEV_ERR_NONFINITE (-5)
#define DEV_ERR_BARRIER (-6)

// A static box in the world frame, FP32 (walls first, then tool boxes).
struct BoxF {
  float c[3];
  float R[9];  // row-major, world = R * local + c
  float h[3];
  int is_tool;
};

// Geometry and material of one scene of a batch (device table; a single
// scene is a batch of one). Scenes never touch: each has its own block of
// broadphase cells, so its particles keep their own coordinates.
constexpr uint32_t kProgStride = 32;  // words between the solver's progress flags

struct SceneGeo {
  float lo[3];                 // origin of the scene's broadphase cells
  int hf_nx, hf_ny;            // heightfield (hf_nx == 0: none)
  float hf_x0, hf_y0, hf_cell;
  uint32_t hf_off;             // first height of the scene in the heights array
  uint32_t box0, nbox, nwall;  // its boxes in the box table, walls first
  float mu_t, mu_tool, mu_r;
  float tp[3], tv[3], tw[3];   // tool motion (point velocity v_T + w_T x (x - p_T))
  int cf, ncx, ncy;            // surface columns of the learned warm start (cf 0: none)
  uint32_t col_off;            // first column of the scene in the surface array
  uint32_t pid0;               // first particle id of the scene (ids are global)
  uint32_t npart;              // its particles (ids pid0 .. pid0 + npart - 1)
  // active-zone cutter (cut_on 0: none), world frame after the tool pose
  int cut_on;
  float e0[3], u[3], ns[3], nf[3];  // edge start, edge direction, blade normal, failure-plane normal
  float cut_len, rho_b, rs, ms, inv_m, inv_I;
};

// Per-step constants, passed by value to every kernel.
struct StepConsts {
  uint32_t n;           // particles (all scenes)
  uint32_t cap;         // contact capacity
  uint32_t nscenes;
  float dt, g[3];
  float ups;            // Upsilon = 1 / (1 + 4 tau / dt), tau = 2 dt
  float estar_pair;     // [2 (1 - nu^2) / E]^-1
  float estar_static;   // E / (1 - nu^2)
  float cohesion;
  int cohesive;
  float sig_t, sig_r;   // gamma_t / dt, gamma_r / dt
  // broadphase: every scene has gnx x gny x gnz cells of width 1/cell_inv
  float cell_inv;
  int gnx, gny, gnz;
  const SceneGeo *geo;
  const BoxF *boxes;    // world-frame boxes of all scenes
  const float *heights; // heightfields of all scenes
};

__device__ __forceinline__ int cell_axis(float x, float x0, float inv, int n) {
  float t = floorf((x - x0) * inv);
  if (!(t >= 0.0f)) return 0;
  if (t >= (float)(n - 1)) return n - 1;
  return (int)t;
}

// Cell of a particle: its scene's block of gnx x gny x gnz cells, then the
// cell inside it (coordinates clamped to the block, which keeps neighbouring
// particles in neighbouring cells). z runs fastest, then y, then x: beds are
// wide and shallow, so slot order walks vertical columns slab by slab and a
// particle's neighbours lie within about one x-slab of it in slot order (the
// solver's CTAs then touch only nearby slot ranges).
__device__ __forceinline__ uint32_t cell_index(const StepConsts &k, const SceneGeo &G, uint32_t sid, float4 p,
                                               int &cx, int &cy, int &cz) {
  cx = cell_axis(p.x, G.lo[0], k.cell_inv, k.gnx);
  cy = cell_axis(p.y, G.lo[1], k.cell_inv, k.gny);
  cz = cell_axis(p.z, G.lo[2], k.cell_inv, k.gnz);
  const uint32_t cps = (uint32_t)k.gnx * (uint32_t)k.gny * (uint32_t)k.gnz;
  return sid * cps + ((uint32_t)cx * (uint32_t)k.gny + (uint32_t)cy) * (uint32_t)k.gnz + (uint32_t)cz;
}


// Device pointers of one scene (passed by value).
struct DevPtrs {
  // particles, slot order (re-sorted by cell every step)
  float4 *pos;                // (x, y, z, r)
  float4 *pv;                 // 32-byte state record per particle: [2i] (v, 1/m), [2i+1] (w, 1/I)
  uint32_t *pid;
  uint32_t *sid;              // scene of the particle
  float4 *pos2, *pv2;         // reorder targets
  uint32_t *pid2, *sid2;
  // grid
  uint32_t *cell_of, *cell_count, *cell_start, *cell_cursor, *perm;
  // contacts in owner order (owner = the particle with the smaller id)
  uint32_t *cnt, *cstart;     // per slot (n + 1)
  uint2 *c_ab;                // slot a, slot b | TDS_STATIC + surface id
  unsigned long long *c_key;
  float4 *c_rn, *c_rq;        // (n, la), (lb, q_n, Sigma_n, f_c)
  float2 *c_rm;               // (mu, rbar mu_r)
  float4 *c_sv, *c_sw;        // static side: point velocity, spin
  float4 *c_la;               // initial impulses (n, t1, t2, r.x)
  float2 *c_lb;               // (r.y, r.z)
  // colouring
  uint32_t *inc_cnt, *inc_start, *inc_cursor;
  uint2 *inc_ent;             // (contact id, high word of its priority) per incidence
  unsigned long long *prio;   // colouring priority per contact
  uint8_t *colour;
  int32_t *wait;
  uint32_t *frontier0, *frontier1;
  // bucketing into colour order
  uint32_t *tile_hist, *tile_off, *order;
  uint32_t *bstart, *bend, *bpad;  // padded colour-order range of each bucket
  uint32_t ntiles;
  // colour order (what the solver streams)
  uint2 *p_ab;
  float4 *p_rn, *p_rq;
  float2 *p_rm;
  float4 *p_sv, *p_sw;
  float4 *p_la;
  float2 *p_lb;
  // warm-start memory by particle id: [0] read, [1] written this step
  uint32_t *prev_first[2], *prev_cnt[2], *prev_other[2];
  float4 *prev_l0[2], *prev_l1[2];
  // scalars and scratch
  uint32_t recolour;          // colour every contact every recolour-th step (1: every step)
  unsigned long long wait_ns; // limit of every wait on other CTAs (grid barriers, neighbour flags)
                              // before the wait gives up and latches DEV_ERR_BARRIER
  int32_t *err;
  uint32_t *ctr;              // see CTR_* below
  unsigned long long *acc;    // see ACC_* below (sums over steps, reset by the host)
  float *fscal;               // see FS_* below
  double *dpart;              // per-block partial sums
  double *dres;               // solver residual: per chunk (numerator, denominator)
  // residual chunks: every (scene, bucket) range of the colour order cut into
  // pieces of at most kResChunk contacts; a chunk holds one scene's contacts
  uint32_t nscenes;           // scenes of the batch
  uint32_t *scq_cnt;          // contacts per (scene, bucket), scene-major
  uint32_t *scq_start;        // colour-order start of each (scene, bucket) range
  uint32_t *scq_chunk;        // first chunk of each (scene, bucket), S * TDS_NBUCKETS + 1
  uint4 *chunk;               // (colour-order start, contacts, scene, 0) per chunk
  float *scene_res;           // per scene: residual at its last check of the last step
  uint32_t *scene_iters;      // per scene: sweeps of the last step
  uint32_t *bar;              // grid barrier: [0] arrivals, [1] generation
  uint32_t *prog;             // solver neighbour sync: last colour phase published per CTA,
                              // one flag per kProgStride words (own 128-byte line)
  uint32_t *rng;              // solver neighbour sync: touched slot range [lo, hi] per CTA
  uint32_t *scan_tmp;
  float *stage;               // 9 n floats for reads
  float *tool_out;            // 6 floats per scene
  double *tool_acc;           // per-scene force and torque accumulators (batches)
  // learned warm start (owner order)
  float *feat;                // 10 features per contact
  float4 *sdirw;              // slip direction s and impulse scale W per contact
  float *targ;                // 3 targets per contact (recording)
  uint8_t *c_flag;            // 1 if the contact's key existed in the previous step
  uint32_t *new_idx;          // learned warm start without recording: the contacts it starts
  // active-zone cut: per heightfield node (all scenes) pending mass, highest
  // height so far, scene, particle count and rank; per particle id the
  // dormant flag/rank and slot
  float *hf_pend, *hf_top;
  uint32_t *hf_scene, *hf_cnt, *hf_rank;
  uint32_t *dorm_rank, *dorm_list, *slot_of_pid;
  float4 *p_il;               // impact stage, colour order: impulses (n, t1, t2, r.x)
  float4 *p_il2;              //   (r.y, r.z, G_n v* before the stage, normal target)
};



enum { CTR_NC = 0, CTR_NCOL = 1, CTR_ITERS = 2, CTR_FCOUNT = 4, /* 4,5,6 */ CTR_NPP = 8,
       CTR_NSTAT = 9, CTR_TOTAL = 10, CTR_ROUNDS = 11, CTR_PADDED = 12, CTR_IMPACTS = 13,
       CTR_NEW = 14, CTR_SPAWN = 15, CTR_CLEAN = 16, CTR_NCHUNK = 17, CTR_COUNT = 18 };
enum { FS_RESID = 0, FS_COUNT = 4 };
// ACC_SWEEP_PP / ACC_SWEEP_ST: sum over steps of sweeps x particle-pair /
// static contacts (the solver's algorithmic work); ACC_STEPS: steps summed.
enum { ACC_SWEEP_PP = 0, ACC_SWEEP_ST = 1, ACC_CONTACTS = 2, ACC_STEPS = 3, ACC_COUNT = 8 };

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }

// One 256-bit access (a single 32-byte sector) for a particle's state
// record, bypassing L1 (other SMs update it between colours).
__device__ __forceinline__ void ld_state(const float4 *rec, float4 &v, float4 &w) {
  asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w), "=f"(w.x), "=f"(w.y), "=f"(w.z), "=f"(w.w)
               : "l"(rec));
}
__device__ __forceinline__ void st_state(float4 *rec, float4 v, float4 w) {
  asm volatile("st.global.cg.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(rec), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w), "f"(w.x), "f"(w.y), "f"(w.z), "f"(w.w)
               : "memory");
}
// Vector arithmetic with every rounding written out (round-to-nearest
// intrinsics, fused multiply-adds where named): the compiler cannot contract
// or reorder them, so a computation rounds the same way in every kernel and
// every instantiation that uses it (the solver's launch shapes give equal
// results bit for bit).
__device__ __forceinline__ float3 operator+(float3 a, float3 b) {
  return make_float3(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z));
}
__device__ __forceinline__ float3 operator-(float3 a, float3 b) {
  return make_float3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}
__device__ __forceinline__ float3 operator*(float s, float3 a) {
  return make_float3(__fmul_rn(s, a.x), __fmul_rn(s, a.y), __fmul_rn(s, a.z));
}
// a + s b, one fused multiply-add per component
__device__ __forceinline__ float3 axpy(float s, float3 b, float3 a) {
  return make_float3(__fmaf_rn(s, b.x, a.x), __fmaf_rn(s, b.y, a.y), __fmaf_rn(s, b.z, a.z));
}
__device__ __forceinline__ float dot(float3 a, float3 b) {
  return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return make_float3(__fmaf_rn(a.y, b.z, -__fmul_rn(a.z, b.y)), __fmaf_rn(a.z, b.x, -__fmul_rn(a.x, b.z)),
                     __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x)));
}

// Orthonormal tangent basis of a unit normal, branch-free (Duff, Burgess,
// Christensen, Hery, Kensler, Liani, Villemin, "Building an Orthonormal
// Basis, Revisited", JCGT 6(1), 2017). The 2-D tangent update is invariant
// under the choice of basis, since its effective mass is isotropic.
__device__ __forceinline__ void onb(float3 n, float3 &t1, float3 &t2) {
  const float sgn = copysignf(1.0f, n.z);
  const float a = -__frcp_rn(__fadd_rn(sgn, n.z));
  const float b = __fmul_rn(__fmul_rn(n.x, n.y), a);
  t1 = make_float3(__fmaf_rn(__fmul_rn(sgn, __fmul_rn(n.x, n.x)), a, 1.0f), __fmul_rn(sgn, b), -__fmul_rn(sgn, n.x));
  t2 = make_float3(b, __fmaf_rn(__fmul_rn(n.y, n.y), a, sgn), -n.y);
}

// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014): the colouring
// priority of a contact key. A bijection, so distinct keys never tie.
__device__ __forceinline__ unsigned long long priority(unsigned long long key) {
  unsigned long long z = key + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// A step that latched an error changes no state from there on, and the
// steps queued after it do nothing: every kernel that writes particle state,
// warm-start memory, the heightfield or the tool force returns at once while
// an error is latched. The state buffers of the failing step's start then
// stay intact for the host to restore.
__device__ __forceinline__ bool step_failed(const DevPtrs &d) { return *(volatile const int32_t *)d.err != 0; }

// Incremental colouring this step: the contacts whose key existed in the
// previous step keep its colour, only the new ones are coloured (every step
// but each recolour-th, counting from the first). The step's index is the
// count of steps that started clean (the broadphase's first kernel counts
// this one), so graph replays take the same decision as launches.
__device__ __forceinline__ bool incremental_colouring(const DevPtrs &d) {
  const uint32_t idx = *(volatile const uint32_t *)(d.ctr + CTR_CLEAN) - 1u;
  return d.recolour > 1u && idx > 0u && idx % d.recolour != 0u;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void latch_error(int32_t *err, int32_t code) {
  atomicCAS(err, 0, code);
}

// Grid-wide barrier for cooperative (co-resident) launches over one arrival
// counter that is zeroed before each launch. gen counts the barriers this
// block has passed (the same for every block): thread 0 adds 1 with release
// semantics (publishing the block's writes, ordered by the preceding
// __syncthreads) without waiting for a reply, then polls with acquire loads
// until the counter reaches (gen + 1) x gridDim.x. The wait is bounded: past
// limit_ns, or when another block latched an error, it returns false
// (latching DEV_ERR_BARRIER on a timeout) in every thread of the block, and
// the caller must return.
__device__ __forceinline__ bool grid_barrier(uint32_t *bar, int32_t *err, uint32_t &gen,
                                             unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    const uint32_t target = (gen + 1u) * gridDim.x;
    int ok = 1;
    unsigned long long t0 = 0;
    for (unsigned spins = 0;; ++spins) {
      uint32_t cur;
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(bar) : "memory");
      if ((int32_t)(cur - target) >= 0) break;
      if ((spins & 31u) == 31u) {
        if (*(volatile int32_t *)err != 0) { ok = 0; break; }
        unsigned long long t = global_ns();
        if (t0 == 0) t0 = t;
        else if (t - t0 > limit_ns) {
          latch_error(err, DEV_ERR_BARRIER);
          ok = 0;
          break;
        }
      }
    }
    if (*(volatile int32_t *)err != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  ++gen;
  return s_ok != 0;
}

// Host-side launchers implemented in the .cu files.
void tds_scan_exclusive(const uint32_t *in, uint32_t *out, uint32_t m, uint32_t *tmp,
                        cudaStream_t st);
size_t tds_scan_tmp_words(uint32_t m);
