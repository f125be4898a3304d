// tds_contacts.cu -- the collision-detection line of Algorithm 1 on the GPU and
// the rows of the contact law for every contact found.
//
//  1. sorted-cell broadphase: bin particles in a uniform grid whose cells are
//     wider than any contact reach, count (atomics), scan (warp shuffles),
//     scatter, sort each cell by particle id, and re-order the particle
//     arrays by cell so that neighbours are contiguous in memory;
//  2. narrowphase per owner particle (the one with the smaller id): the 27
//     cells around it as 9 runs of 3 cells contiguous along z (the fastest
//     axis of the cell order), the heightfield triangle under
//     it and every wall / tool box, each decided by the FP32 predicate below,
//     which is bit-identical to the CPU oracle's (explicit round-to-nearest
//     intrinsics, no FMA contraction);
//  3. per contact, in FP32: normal, overlap, lever arms, Hertz stiffness
//     k_n = E* sqrt(d*)/3 mapped onto the SPOOK normal row (unit-Jacobian
//     form: Sigma_n = (4/dt^2) Upsilon 4/(5 k_n sqrt(delta)),
//     q_n = -(4/dt) Upsilon g + Upsilon G v_n with g = -(4/5) delta), the
//     cohesion bound dt c_p pi rbar^2, friction and rolling bounds, and the
//     warm-start impulses of the same contact key from the previous step.
#include "tds_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// FP32 predicates: the bit-exact contract with the oracle
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool pp_touch(float4 A, float4 B, int cohesive) {
  float dx = __fsub_rn(B.x, A.x), dy = __fsub_rn(B.y, A.y), dz = __fsub_rn(B.z, A.z);
  float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  float rs = __fadd_rn(A.w, B.w);
  float R = cohesive ? __fadd_rn(rs, __fmul_rn(0.025f, rs)) : rs;
  return d2 < __fmul_rn(R, R);
}

__device__ __forceinline__ float static_reach(float r, int cohesive) {
  return cohesive ? __fadd_rn(r, __fmul_rn(0.025f, __fadd_rn(r, r))) : r;
}

struct HfHit {
  float s;       // signed distance of the centre from the triangle's plane
  float a, b;    // height differences along the two legs from the base vertex
  float den;     // sqrt(cell^2 + a^2 + b^2)
  int upper;
};

__device__ __forceinline__ HfHit hf_distance(const SceneGeo &G, const float *heights, float px, float py,
                                             float pz) {
  const int nx = G.hf_nx, ny = G.hf_ny, stride = nx + 1;
  float tx = __fdiv_rn(__fsub_rn(px, G.hf_x0), G.hf_cell);
  float ty = __fdiv_rn(__fsub_rn(py, G.hf_y0), G.hf_cell);
  float fx = floorf(tx), fy = floorf(ty);
  int i, j;
  if (!(fx >= 0.0f)) i = 0; else if (fx > (float)(nx - 1)) i = nx - 1; else i = (int)fx;
  if (!(fy >= 0.0f)) j = 0; else if (fy > (float)(ny - 1)) j = ny - 1; else j = (int)fy;
  float u = __fsub_rn(tx, (float)i), v = __fsub_rn(ty, (float)j);
  const float *h = heights + G.hf_off;
  HfHit r;
  float hb, uu, vv;
  r.upper = !(__fadd_rn(u, v) <= 1.0f);
  if (!r.upper) {
    hb = __ldg(h + j * stride + i);
    r.a = __fsub_rn(__ldg(h + j * stride + i + 1), hb);
    r.b = __fsub_rn(__ldg(h + (j + 1) * stride + i), hb);
    uu = u; vv = v;
  } else {
    hb = __ldg(h + (j + 1) * stride + i + 1);
    r.a = __fsub_rn(__ldg(h + (j + 1) * stride + i), hb);
    r.b = __fsub_rn(__ldg(h + j * stride + i + 1), hb);
    uu = __fsub_rn(1.0f, u); vv = __fsub_rn(1.0f, v);
  }
  float e = __fsub_rn(pz, hb);
  e = __fsub_rn(e, __fmul_rn(r.a, uu));
  e = __fsub_rn(e, __fmul_rn(r.b, vv));
  float num = __fmul_rn(G.hf_cell, e);
  r.den = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(G.hf_cell, G.hf_cell), __fmul_rn(r.a, r.a)),
                               __fmul_rn(r.b, r.b)));
  r.s = __fdiv_rn(num, r.den);
  return r;
}

struct BoxHit {
  float l[3], e[3];
  float d2;
};

__device__ __forceinline__ BoxHit box_distance(const BoxF &B, float px, float py, float pz) {
  BoxHit r;
  float dx = __fsub_rn(px, B.c[0]), dy = __fsub_rn(py, B.c[1]), dz = __fsub_rn(pz, B.c[2]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.l[k] = __fadd_rn(__fadd_rn(__fmul_rn(B.R[k], dx), __fmul_rn(B.R[3 + k], dy)),
                       __fmul_rn(B.R[6 + k], dz));
    float q = fminf(fmaxf(r.l[k], -B.h[k]), B.h[k]);
    r.e[k] = __fsub_rn(r.l[k], q);
  }
  r.d2 = __fadd_rn(__fadd_rn(__fmul_rn(r.e[0], r.e[0]), __fmul_rn(r.e[1], r.e[1])),
                   __fmul_rn(r.e[2], r.e[2]));
  return r;
}

// ---------------------------------------------------------------------------
// broadphase kernels
// ---------------------------------------------------------------------------
// Dormant reserve slots (radius 0) go to one trailing cell after all scenes'
// cells, which no neighbour search visits.
__global__ void k_cells(DevPtrs d, StepConsts k) {
  // steps that start with no error latched (the host finds a failing step by it)
  if (blockIdx.x == 0 && threadIdx.x == 0 && !step_failed(d)) atomicAdd(d.ctr + CTR_CLEAN, 1u);
  const uint32_t trailing = k.nscenes * (uint32_t)k.gnx * (uint32_t)k.gny * (uint32_t)k.gnz;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n; i += gridDim.x * blockDim.x) {
    int cx, cy, cz;
    const uint32_t sid = d.sid[i];
    const float4 P = d.pos[i];
    uint32_t c = P.w == 0.0f ? trailing : cell_index(k, k.geo[sid], sid, P, cx, cy, cz);
    d.cell_of[i] = c;
    atomicAdd(d.cell_count + c, 1u);
  }
}

__global__ void k_cell_scatter(DevPtrs d, StepConsts k) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n; i += gridDim.x * blockDim.x) {
    uint32_t dst = atomicAdd(d.cell_cursor + d.cell_of[i], 1u);
    d.perm[dst] = i;
  }
}

// Sort each cell's entries by particle id so the order is reproducible
// (cells hold a handful of particles; crowded border cells are left as is).
__global__ void k_cell_sort(DevPtrs d, uint32_t ncells) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    uint32_t s = d.cell_start[c], e = d.cell_start[c + 1];
    if (e - s < 2 || e - s > 64) continue;
    for (uint32_t a = s + 1; a < e; ++a) {
      uint32_t v = d.perm[a], key = d.pid[v];
      uint32_t b = a;
      while (b > s && d.pid[d.perm[b - 1]] > key) { d.perm[b] = d.perm[b - 1]; --b; }
      d.perm[b] = v;
    }
  }
}

__global__ void k_reorder(DevPtrs d, uint32_t n) {
  if (step_failed(d)) return;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    uint32_t i = d.perm[j];
    d.pos2[j] = d.pos[i];
    reinterpret_cast<double4 *>(d.pv2)[j] = reinterpret_cast<const double4 *>(d.pv)[i];
    d.pid2[j] = d.pid[i];
    d.sid2[j] = d.sid[i];
  }
}

// ---------------------------------------------------------------------------
// narrowphase
// ---------------------------------------------------------------------------
// Calls f.pair(j, pid_j, Q), f.hf(hit), f.box(b, hit) for every contact owned
// by slot i, in a fixed order.
template <class F>
__device__ __forceinline__ void for_each_contact(const DevPtrs &d, const StepConsts &k, uint32_t i, F &f) {
  const float4 P = d.pos[i];
  if (P.w == 0.0f) return;  // dormant reserve slot: no contacts
  const uint32_t me = d.pid[i], sid = d.sid[i];
  const SceneGeo &G = k.geo[sid];
  int cx, cy, cz;
  (void)cell_index(k, G, sid, P, cx, cy, cz);
  const uint32_t block = sid * (uint32_t)k.gnx * (uint32_t)k.gny * (uint32_t)k.gnz;
  const int z0 = max(cz - 1, 0), z1 = min(cz + 1, k.gnz - 1);
  for (int x = max(cx - 1, 0); x <= min(cx + 1, k.gnx - 1); ++x) {
    for (int y = max(cy - 1, 0); y <= min(cy + 1, k.gny - 1); ++y) {
      uint32_t row = block + ((uint32_t)x * (uint32_t)k.gny + (uint32_t)y) * (uint32_t)k.gnz;
      uint32_t s = __ldg(d.cell_start + row + z0), e = __ldg(d.cell_start + row + z1 + 1);
      for (uint32_t j = s; j < e; ++j) {
        uint32_t pj = __ldg(d.pid + j);
        if (pj <= me) continue;
        float4 Q = __ldg(d.pos + j);
        if (pp_touch(P, Q, k.cohesive)) f.pair(j, pj, Q);
      }
    }
  }
  if (G.hf_nx > 0) {
    HfHit hit = hf_distance(G, k.heights, P.x, P.y, P.z);
    if (hit.s < static_reach(P.w, k.cohesive)) f.hf(G, hit);
  }
  for (uint32_t b = 0; b < G.nbox; ++b) {
    const BoxF &B = k.boxes[G.box0 + b];
    float reach = static_reach(P.w, k.cohesive && !B.is_tool);
    BoxHit hit = box_distance(B, P.x, P.y, P.z);
    if (hit.d2 < __fmul_rn(reach, reach)) f.box(G, B, b, hit);
  }
}

struct Counter {
  uint32_t n = 0;
  __device__ void pair(uint32_t, uint32_t, float4) { ++n; }
  __device__ void hf(const SceneGeo &, const HfHit &) { ++n; }
  __device__ void box(const SceneGeo &, const BoxF &, uint32_t, const BoxHit &) { ++n; }
};

__global__ void k_count(DevPtrs d, StepConsts k) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n; i += gridDim.x * blockDim.x) {
    Counter c;
    for_each_contact(d, k, i, c);
    d.cnt[i] = c.n;
  }
}

__global__ void k_total(DevPtrs d, StepConsts k) {
  uint32_t total = d.cstart[k.n];
  d.ctr[CTR_TOTAL] = total;
  d.ctr[CTR_NC] = total < k.cap ? total : k.cap;
  if (total > k.cap) latch_error(d.err, DEV_ERR_CAPACITY);
}

struct Writer {
  const DevPtrs &d;
  const StepConsts &k;
  uint32_t i, me, next;
  float4 P, Va;
  int use_prev;
  uint32_t pf, pc;
  bool inc;  // incremental colouring: contacts of a previous key keep its colour

  // Common part of every contact: rows and warm start. n points from a
  // towards b (into a static surface), delta is the overlap, vb/wb the other
  // side's velocity at the start of the step.
  __device__ void emit(const SceneGeo &G, uint32_t b_slot, uint32_t other, float3 n, float delta,
                       float rb, float dstar, float estar, float rbar, float dfloor, bool is_static,
                       bool is_tool, float3 vb, float3 vs, float3 ws) {
    uint32_t c = next++;
    if (c >= k.cap) return;
    const float h = k.dt;
    float la = P.w - 0.5f * delta;
    float lb = is_static ? 0.0f : rb - 0.5f * delta;
    float kn = estar * sqrtf(dstar) * (1.0f / 3.0f);
    float ds = fmaxf(delta, dfloor);
    float eps = 4.0f / (5.0f * kn * sqrtf(ds));
    float Sn = 4.0f / (h * h) * k.ups * eps;
    float g = -0.8f * delta;
    float Jv0 = dot(n, vb - f3(Va));
    float qn = -4.0f / h * k.ups * g + k.ups * Jv0;
    float fc = (k.cohesive && !is_tool) ? h * k.cohesion * 3.14159265358979f * rbar * rbar : 0.0f;
    float mu = is_tool ? G.mu_tool : G.mu_t;
    float rmu = rbar * G.mu_r;
    unsigned long long key = ((unsigned long long)me << 32) | other;
    d.c_ab[c] = make_uint2(i, b_slot);
    d.c_key[c] = key;
    // colouring priority of the scene-local key: a scene of a batch is
    // coloured exactly as it is alone
    const uint32_t lo = is_static ? other : other - G.pid0;
    d.prio[c] = priority(((unsigned long long)(me - G.pid0) << 32) | lo);
    d.c_rn[c] = make_float4(n.x, n.y, n.z, la);
    d.c_rq[c] = make_float4(lb, qn, Sn, fc);
    d.c_rm[c] = make_float2(mu, rmu);
    if (is_static) {
      d.c_sv[c] = make_float4(vs.x, vs.y, vs.z, 0.0f);
      d.c_sw[c] = make_float4(ws.x, ws.y, ws.z, 0.0f);
    }
    // warm start: previous impulses of the same key, tangent re-projected
    // onto the new tangent plane, everything clamped into the new bounds
    float4 la0 = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 lb0 = make_float2(0.f, 0.f);
    uint8_t persisted = 0;
    uint32_t kept = TDS_NO_COLOUR;
    if (use_prev || inc) {
      for (uint32_t q = pf; q < pf + pc; ++q) {
        if (__ldg(d.prev_other[0] + q) != other) continue;
        float4 l0 = d.prev_l0[0][q], l1 = d.prev_l1[0][q];
        kept = __float_as_uint(l1.w);  // the key's colour in the previous step
        if (!use_prev) break;
        float ln = fmaxf(l0.x, -fc);
        float3 t1, t2;
        onb(n, t1, t2);
        float3 tw = make_float3(l0.y, l0.z, l0.w);
        float a1 = dot(t1, tw), a2 = dot(t2, tw);
        float bt = mu * fabsf(ln), m2 = sqrtf(a1 * a1 + a2 * a2);
        if (m2 > bt) { float s = bt > 0.f ? bt / m2 : 0.f; a1 *= s; a2 *= s; }
        float3 lr = make_float3(l1.x, l1.y, l1.z);
        float br = rmu * fabsf(ln), mr = sqrtf(dot(lr, lr));
        if (mr > br) lr = (br > 0.f ? br / mr : 0.f) * lr;
        la0 = make_float4(ln, a1, a2, lr.x);
        lb0 = make_float2(lr.y, lr.z);
        persisted = 1;
        break;
      }
    }
    d.c_la[c] = la0;
    d.c_lb[c] = lb0;
    d.c_flag[c] = persisted;
    if (inc) d.colour[c] = (uint8_t)(kept < TDS_MAX_COLOURS ? kept : TDS_NO_COLOUR);
  }

  __device__ void pair(uint32_t j, uint32_t pj, float4 Q) {
    float3 dv = f3(Q) - f3(P);
    float dist = sqrtf(dot(dv, dv));
    float3 n = dist > 0.0f ? (1.0f / dist) * dv : make_float3(0.f, 0.f, 1.f);
    float delta = P.w + Q.w - dist;
    float rs = P.w + Q.w;
    float dstar = 2.0f * P.w * Q.w / rs;
    float4 Vb = d.pv[2 * j];
    float3 z3 = make_float3(0.f, 0.f, 0.f);
    emit(k.geo[d.sid[i]], j, pj, n, delta, Q.w, dstar, k.estar_pair, dstar, 1e-5f * rs, false, false,
         f3(Vb), z3, z3);
  }

  __device__ void surface(const SceneGeo &G, uint32_t surf, float3 ns, float s, bool is_tool) {
    float3 n = make_float3(-ns.x, -ns.y, -ns.z);
    float delta = P.w - s;
    float3 vs = make_float3(0.f, 0.f, 0.f), ws = vs;
    if (is_tool) {
      float la = P.w - 0.5f * delta;
      float3 xc = f3(P) + la * n;
      float3 rel = xc - make_float3(G.tp[0], G.tp[1], G.tp[2]);
      ws = make_float3(G.tw[0], G.tw[1], G.tw[2]);
      vs = make_float3(G.tv[0], G.tv[1], G.tv[2]) + cross(ws, rel);
    }
    emit(G, TDS_STATIC | surf, TDS_STATIC | surf, n, delta, 0.f, 2.0f * P.w, k.estar_static, P.w,
         2e-5f * P.w, true, is_tool, vs, vs, ws);
  }

  __device__ void hf(const SceneGeo &G, const HfHit &hit) {
    float inv = 1.0f / hit.den;
    float3 ns = hit.upper ? make_float3(hit.a * inv, hit.b * inv, G.hf_cell * inv)
                          : make_float3(-hit.a * inv, -hit.b * inv, G.hf_cell * inv);
    surface(G, 0u, ns, hit.s, false);
  }

  __device__ void box(const SceneGeo &G, const BoxF &B, uint32_t b, const BoxHit &hit) {
    float3 ns;
    float s;
    if (hit.d2 > 0.0f) {
      s = sqrtf(hit.d2);
      float inv = 1.0f / s;
      ns = make_float3((B.R[0] * hit.e[0] + B.R[1] * hit.e[1] + B.R[2] * hit.e[2]) * inv,
                       (B.R[3] * hit.e[0] + B.R[4] * hit.e[1] + B.R[5] * hit.e[2]) * inv,
                       (B.R[6] * hit.e[0] + B.R[7] * hit.e[1] + B.R[8] * hit.e[2]) * inv);
    } else {
      int ax = 0;
      float depth = B.h[0] - fabsf(hit.l[0]);
      for (int m = 1; m < 3; ++m) {
        float dm = B.h[m] - fabsf(hit.l[m]);
        if (dm < depth) { depth = dm; ax = m; }
      }
      float side = hit.l[ax] >= 0.0f ? 1.0f : -1.0f;
      s = -depth;
      ns = make_float3(side * B.R[ax], side * B.R[3 + ax], side * B.R[6 + ax]);
    }
    surface(G, 1u + b, ns, s, B.is_tool != 0);
  }
};

__global__ void k_write(DevPtrs d, StepConsts k, int use_prev) {
  const bool inc = incremental_colouring(d);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n; i += gridDim.x * blockDim.x) {
    Writer w{d, k, i, d.pid[i], d.cstart[i], d.pos[i], d.pv[2 * i], use_prev, 0u, 0u, inc};
    if (use_prev || inc) {
      w.pf = d.prev_first[0][w.me];
      w.pc = d.prev_cnt[0][w.me];
    }
    for_each_contact(d, k, i, w);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static inline unsigned grid_for(uint32_t n, unsigned threads, unsigned maxb = 152 * 16) {
  unsigned b = (unsigned)((n + threads - 1) / threads);
  if (b == 0) b = 1;
  return b < maxb ? b : maxb;
}

int tds_launch_broadphase(const DevPtrs &d, const StepConsts &k, uint32_t ncells, cudaStream_t st) {
  // ncells scene cells plus the trailing cell of dormant slots
  cudaMemsetAsync(d.cell_count, 0, sizeof(uint32_t) * (ncells + 2), st);
  k_cells<<<grid_for(k.n, 256), 256, 0, st>>>(d, k);
  tds_scan_exclusive(d.cell_count, d.cell_start, ncells + 1, d.scan_tmp, st);
  cudaMemcpyAsync(d.cell_cursor, d.cell_start, sizeof(uint32_t) * (ncells + 1), cudaMemcpyDeviceToDevice, st);
  k_cell_scatter<<<grid_for(k.n, 256), 256, 0, st>>>(d, k);
  k_cell_sort<<<grid_for(ncells, 256), 256, 0, st>>>(d, ncells);
  k_reorder<<<grid_for(k.n, 256), 256, 0, st>>>(d, k.n);
  return 8;
}

// After the reorder (pointers swapped by the caller): count, scan, write.
int tds_launch_narrowphase(const DevPtrs &d, const StepConsts &k, int use_prev, cudaStream_t st) {
  k_count<<<grid_for(k.n, 128), 128, 0, st>>>(d, k);
  tds_scan_exclusive(d.cnt, d.cstart, k.n, d.scan_tmp, st);
  k_total<<<1, 1, 0, st>>>(d, k);
  k_write<<<grid_for(k.n, 128), 128, 0, st>>>(d, k, use_prev);
  return 6;
}
