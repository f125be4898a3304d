// tds_solve.cu -- "solve the mesoscale MCP using iterative PGS solver" and
// "update positions" of Algorithm 1.
//
// The MCP of the SPOOK stepper (section "Contacting rigid multibodies") is
// solved by projected Gauss-Seidel on the physical impulses, colour by
// colour: within a colour no two contacts share a particle, so all of them
// are updated in parallel and the result equals sequential Gauss-Seidel in
// colour-major order. One persistent, co-resident kernel runs the whole
// solve with a grid barrier between colours: first v = M^-1 (p + G^T
// lambda_0) from the warm-start impulses, then the sweeps. Per contact and
// sweep: the normal row (clamped at -f_c), the 2-D tangent rows projected on
// the Coulomb disk mu |Lambda_n|, the 3 rolling rows projected on the ball
// rbar mu_r |Lambda_n| (Eqs. signCoul1-3), each followed by
// v += M^-1 G^T dLambda. Particle velocities are read and written through L2
// (ld.global.cg / st.global.cg) because other SMs update them between colours.
#include "tds_internal.cuh"

namespace {

__device__ __forceinline__ bool is_dyn(uint32_t b) { return (b & TDS_STATIC) == 0u; }

__global__ void k_predict(DevPtrs d, StepConsts k) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n; i += gridDim.x * blockDim.x) {
    float4 v = d.vel[i];
    v.x += k.dt * k.g[0];
    v.y += k.dt * k.g[1];
    v.z += k.dt * k.g[2];
    d.vel[i] = v;
  }
}

struct Side {
  float3 v, w;
  float im, iI;
};

__device__ __forceinline__ Side load_side(const DevPtrs &d, uint32_t s) {
  float4 v = __ldcg(d.vel + s), w = __ldcg(d.ang + s);
  return Side{f3(v), f3(w), v.w, w.w};
}
__device__ __forceinline__ void store_side(const DevPtrs &d, uint32_t s, const Side &x) {
  __stcg(d.vel + s, make_float4(x.v.x, x.v.y, x.v.z, x.im));
  __stcg(d.ang + s, make_float4(x.w.x, x.w.y, x.w.z, x.iI));
}

struct Row {
  uint2 ab;
  float3 n;
  float la, lb, qn, Sn, fc, mu, rmu;
  float3 sv, sw;
  bool dyn;
};

__device__ __forceinline__ Row load_row(const DevPtrs &d, uint32_t p) {
  Row r;
  r.ab = d.p_ab[p];
  float4 rn = d.p_rn[p], rq = d.p_rq[p];
  float2 rm = d.p_rm[p];
  r.n = f3(rn);
  r.la = rn.w;
  r.lb = rq.x; r.qn = rq.y; r.Sn = rq.z; r.fc = rq.w;
  r.mu = rm.x; r.rmu = rm.y;
  r.dyn = is_dyn(r.ab.y);
  if (!r.dyn) { r.sv = f3(d.p_sv[p]); r.sw = f3(d.p_sw[p]); }
  return r;
}

__device__ __forceinline__ void disk(float &a, float &b, float bound) {
  float m = sqrtf(a * a + b * b);
  if (m > bound) { float s = bound > 0.f ? bound / m : 0.f; a *= s; b *= s; }
}
__device__ __forceinline__ void ball(float3 &a, float bound) {
  float m = sqrtf(dot(a, a));
  if (m > bound) a = (bound > 0.f ? bound / m : 0.f) * a;
}

// v += M^-1 G^T (dn, dt(world), dr) on both sides.
__device__ __forceinline__ void apply(const Row &r, Side &A, Side &B, float dn, float3 dt, float3 dr) {
  float3 P = dn * r.n + dt;
  A.v = A.v - A.im * P;
  A.w = A.w - A.iI * (cross(r.la * r.n, dt) + dr);
  if (r.dyn) {
    B.v = B.v + B.im * P;
    B.w = B.w + B.iI * (cross((-r.lb) * r.n, dt) + dr);
  }
}

__device__ __forceinline__ float3 slip(const Row &r, const Side &A, const Side &B) {
  return (B.v + cross(B.w, (-r.lb) * r.n)) - (A.v + cross(A.w, r.la * r.n));
}

// One projected Gauss-Seidel update of one contact.
__device__ __forceinline__ void pgs_update(const Row &r, Side &A, Side &B, float4 &L0, float2 &L1,
                                           float sig_t, float sig_r) {
  const float3 z3 = make_float3(0.f, 0.f, 0.f);
  // normal row
  float Dn = A.im + B.im + r.Sn;
  float res = dot(r.n, B.v - A.v) + r.Sn * L0.x - r.qn;
  float ln = fmaxf(L0.x - res / Dn, -r.fc);
  float dln = ln - L0.x;
  L0.x = ln;
  apply(r, A, B, dln, z3, z3);
  // tangent rows (Coulomb disk)
  float3 t1, t2;
  onb(r.n, t1, t2);
  float Dt = A.im + B.im + r.la * r.la * A.iI + r.lb * r.lb * B.iI + sig_t;
  float3 u = slip(r, A, B);
  float y1 = L0.y - (dot(t1, u) + sig_t * L0.y) / Dt;
  float y2 = L0.z - (dot(t2, u) + sig_t * L0.z) / Dt;
  disk(y1, y2, r.mu * fabsf(ln));
  float3 dt = (y1 - L0.y) * t1 + (y2 - L0.z) * t2;
  L0.y = y1; L0.z = y2;
  apply(r, A, B, 0.f, dt, z3);
  // rolling rows (ball)
  float Dr = A.iI + B.iI + sig_r;
  float3 lr = make_float3(L0.w, L1.x, L1.y);
  float3 y = lr - (1.0f / Dr) * ((B.w - A.w) + sig_r * lr);
  ball(y, r.rmu * fabsf(ln));
  float3 dr = y - lr;
  L0.w = y.x; L1.x = y.y; L1.y = y.z;
  apply(r, A, B, 0.f, z3, dr);
}

// Contribution of one contact to the natural-map residual (Jacobi pass).
__device__ __forceinline__ void resid_terms(const Row &r, const Side &A, const Side &B, float4 L0,
                                            float2 L1, float sig_t, float sig_r, double &num,
                                            double &den) {
  float Dn = A.im + B.im + r.Sn;
  float wn = dot(r.n, B.v - A.v) + r.Sn * L0.x - r.qn;
  float pn = fmaxf(L0.x - wn / Dn, -r.fc);
  float3 t1, t2;
  onb(r.n, t1, t2);
  float Dt = A.im + B.im + r.la * r.la * A.iI + r.lb * r.lb * B.iI + sig_t;
  float3 u = slip(r, A, B);
  float y1 = L0.y - (dot(t1, u) + sig_t * L0.y) / Dt;
  float y2 = L0.z - (dot(t2, u) + sig_t * L0.z) / Dt;
  disk(y1, y2, r.mu * fabsf(L0.x));
  float Dr = A.iI + B.iI + sig_r;
  float3 lr = make_float3(L0.w, L1.x, L1.y);
  float3 y = lr - (1.0f / Dr) * ((B.w - A.w) + sig_r * lr);
  ball(y, r.rmu * fabsf(L0.x));
  float e0 = L0.x - pn, e1 = L0.y - y1, e2 = L0.z - y2;
  float3 e3 = lr - y;
  num += (double)(e0 * e0 + e1 * e1 + e2 * e2 + dot(e3, e3));
  den += (double)(L0.x * L0.x + L0.y * L0.y + L0.z * L0.z + dot(lr, lr));
}

__device__ __forceinline__ void load_pair(const DevPtrs &d, const Row &r, Side &A, Side &B) {
  A = load_side(d, r.ab.x);
  if (r.dyn) B = load_side(d, r.ab.y);
  else B = Side{r.sv, r.sw, 0.f, 0.f};
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  __syncthreads();
  return t;  // valid in thread 0
}

struct SolveArgs {
  uint32_t max_iters, every;
  float tol, sig_t, sig_r;
  int apply_warm;
};

__global__ void __launch_bounds__(256) k_pgs(DevPtrs d, SolveArgs a) {
  __shared__ double sh[8];
  __shared__ int s_stop;
  const uint32_t ncol = d.ctr[CTR_NCOL];
  const uint32_t nc = d.ctr[CTR_NC];
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  // v = M^-1 (p + G^T lambda_0), colour by colour (no conflicts inside one)
  if (a.apply_warm) {
    for (uint32_t col = 0; col < ncol; ++col) {
      const uint32_t s = d.bucket_start[2 * col], e = d.bucket_start[2 * col + 2];
      for (uint32_t p = s + tid; p < e; p += stride) {
        float4 L0 = d.p_la[p];
        float2 L1 = d.p_lb[p];
        if (L0.x == 0.f && L0.y == 0.f && L0.z == 0.f && L0.w == 0.f && L1.x == 0.f && L1.y == 0.f)
          continue;
        Row r = load_row(d, p);
        Side A, B;
        load_pair(d, r, A, B);
        float3 t1, t2;
        onb(r.n, t1, t2);
        apply(r, A, B, L0.x, L0.y * t1 + L0.z * t2, make_float3(L0.w, L1.x, L1.y));
        store_side(d, r.ab.x, A);
        if (r.dyn) store_side(d, r.ab.y, B);
      }
      if (!grid_barrier(d.bar, d.err)) return;
    }
  }
  uint32_t it = 0;
  float resid = -1.f;
  while (it < a.max_iters) {
    for (uint32_t col = 0; col < ncol; ++col) {
      const uint32_t s = d.bucket_start[2 * col], e = d.bucket_start[2 * col + 2];
      for (uint32_t p = s + tid; p < e; p += stride) {
        Row r = load_row(d, p);
        float4 L0 = d.p_la[p];
        float2 L1 = d.p_lb[p];
        Side A, B;
        load_pair(d, r, A, B);
        pgs_update(r, A, B, L0, L1, a.sig_t, a.sig_r);
        store_side(d, r.ab.x, A);
        if (r.dyn) store_side(d, r.ab.y, B);
        d.p_la[p] = L0;
        d.p_lb[p] = L1;
      }
      if (!grid_barrier(d.bar, d.err)) return;
    }
    ++it;
    if (it == a.max_iters || (a.tol > 0.f && it % a.every == 0)) {
      double num = 0.0, den = 0.0;
      for (uint32_t p = tid; p < nc; p += stride) {
        Row r = load_row(d, p);
        Side A, B;
        load_pair(d, r, A, B);
        resid_terms(r, A, B, __ldcg(d.p_la + p), __ldcg(d.p_lb + p), a.sig_t, a.sig_r, num, den);
      }
      double bn = block_sum(num, sh);
      double bd = block_sum(den, sh);
      if (threadIdx.x == 0) {
        __stcg(d.dpart + 2 * blockIdx.x, bn);
        __stcg(d.dpart + 2 * blockIdx.x + 1, bd);
      }
      if (!grid_barrier(d.bar, d.err)) return;
      if (threadIdx.x == 0) {
        double tn = 0.0, td = 0.0;
        for (uint32_t b = 0; b < gridDim.x; ++b) {
          tn += __ldcg(d.dpart + 2 * b);
          td += __ldcg(d.dpart + 2 * b + 1);
        }
        resid = (float)(sqrt(tn) / fmax(sqrt(td), 1e-12));
        s_stop = a.tol > 0.f && resid <= a.tol;
      }
      __syncthreads();
      if (s_stop) break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.ctr[CTR_ITERS] = it;
    d.fscal[FS_RESID] = resid;
    uint32_t nst = 0;
    for (uint32_t c = 0; c < ncol; ++c) nst += d.bucket_start[2 * c + 2] - d.bucket_start[2 * c + 1];
    d.acc[ACC_SWEEP_PP] += (unsigned long long)it * (nc - nst);
    d.acc[ACC_SWEEP_ST] += (unsigned long long)it * nst;
    d.acc[ACC_CONTACTS] += nc;
    d.acc[ACC_STEPS] += 1;
  }
}

// Colour order -> owner order warm-start memory: (key's other side,
// impulses with the tangent in world coordinates); per particle id the range
// of its owned contacts.
__global__ void k_writeback(DevPtrs d) {
  const uint32_t nc = d.ctr[CTR_NC];
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nc; p += gridDim.x * blockDim.x) {
    uint32_t c = d.order[p];
    float4 L0 = d.p_la[p];
    float2 L1 = d.p_lb[p];
    float3 n = f3(d.p_rn[p]), t1, t2;
    onb(n, t1, t2);
    float3 tw = L0.y * t1 + L0.z * t2;
    d.prev_other[1][c] = (uint32_t)(d.c_key[c] & 0xFFFFFFFFull);
    d.prev_l0[1][c] = make_float4(L0.x, tw.x, tw.y, tw.z);
    d.prev_l1[1][c] = make_float4(L0.w, L1.x, L1.y, 0.f);
  }
}

__global__ void k_prev_ranges(DevPtrs d, uint32_t n, uint32_t cap) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t s = d.cstart[i], e = d.cstart[i + 1];
    if (s > cap) s = cap;
    if (e > cap) e = cap;
    uint32_t me = d.pid[i];
    d.prev_first[1][me] = s;
    d.prev_cnt[1][me] = e - s;
  }
}

__global__ void k_integrate(DevPtrs d, StepConsts k) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n; i += gridDim.x * blockDim.x) {
    float4 p = d.pos[i], v = d.vel[i], w = d.ang[i];
    p.x += k.dt * v.x;
    p.y += k.dt * v.y;
    p.z += k.dt * v.z;
    d.pos[i] = p;
    if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(v.x) && isfinite(v.y) &&
          isfinite(v.z) && isfinite(w.x) && isfinite(w.y) && isfinite(w.z)))
      latch_error(d.err, DEV_ERR_NONFINITE);
  }
}

// Soil-on-tool force and torque about the tool origin: sum over tool
// contacts of (Lambda_n n + Lambda_t) / dt at the contact point, plus the
// rolling impulse / dt. Fixed block partition + fixed-order sums: the
// result is reproducible.
constexpr int kToolBlocks = 128;
__global__ void k_tool_partial(DevPtrs d, StepConsts k) {
  __shared__ double sh[8];
  const uint32_t nc = d.ctr[CTR_NC];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const uint32_t first_tool = 1u + (uint32_t)k.n_walls;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nc; p += gridDim.x * blockDim.x) {
    uint2 ab = d.p_ab[p];
    if (is_dyn(ab.y) || (ab.y & ~TDS_STATIC) < first_tool) continue;
    float4 rn = d.p_rn[p], L0 = d.p_la[p];
    float2 L1 = d.p_lb[p];
    float3 n = f3(rn), t1, t2;
    onb(n, t1, t2);
    float3 F = (1.0f / k.dt) * (L0.x * n + L0.y * t1 + L0.z * t2);
    float3 xc = f3(d.pos[ab.x]) + rn.w * n;
    float3 arm = xc - make_float3(k.tp[0], k.tp[1], k.tp[2]);
    float3 T = cross(arm, F) + (1.0f / k.dt) * make_float3(L0.w, L1.x, L1.y);
    acc[0] += F.x; acc[1] += F.y; acc[2] += F.z;
    acc[3] += T.x; acc[4] += T.y; acc[5] += T.z;
  }
  for (int q = 0; q < 6; ++q) {
    double t = block_sum(acc[q], sh);
    if (threadIdx.x == 0) d.dpart[6 * blockIdx.x + q] = t;
  }
}

__global__ void k_tool_final(DevPtrs d) {
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int b = 0; b < kToolBlocks; ++b) t += d.dpart[6 * b + threadIdx.x];
    d.tool_out[threadIdx.x] = (float)t;
  }
}

// slot order -> particle-id order staging: x y z vx vy vz wx wy wz
__global__ void k_stage(DevPtrs d, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t id = d.pid[i];
    float4 p = d.pos[i], v = d.vel[i], w = d.ang[i];
    d.stage[0 * (size_t)n + id] = p.x; d.stage[1 * (size_t)n + id] = p.y;
    d.stage[2 * (size_t)n + id] = p.z; d.stage[3 * (size_t)n + id] = v.x;
    d.stage[4 * (size_t)n + id] = v.y; d.stage[5 * (size_t)n + id] = v.z;
    d.stage[6 * (size_t)n + id] = w.x; d.stage[7 * (size_t)n + id] = w.y;
    d.stage[8 * (size_t)n + id] = w.z;
  }
}

}  // namespace

static inline unsigned grid_for(uint32_t n, unsigned threads, unsigned maxb = 152 * 16) {
  unsigned b = (unsigned)((n + threads - 1) / threads);
  if (b == 0) b = 1;
  return b < maxb ? b : maxb;
}

int tds_launch_predict(const DevPtrs &d, const StepConsts &k, cudaStream_t st) {
  k_predict<<<grid_for(k.n, 256), 256, 0, st>>>(d, k);
  return 1;
}

cudaError_t tds_launch_pgs(const DevPtrs &d, const StepConsts &k, uint32_t max_iters, float tol,
                           uint32_t every, int apply_warm, int blocks, cudaStream_t st) {
  SolveArgs a{max_iters, every ? every : 1u, tol, k.sig_t, k.sig_r, apply_warm};
  cudaMemsetAsync(d.bar, 0, 2 * sizeof(uint32_t), st);
  DevPtrs dd = d;
  void *args[] = {&dd, &a};
  return cudaLaunchCooperativeKernel((const void *)k_pgs, dim3(blocks), dim3(256), args, 0, st);
}

int tds_launch_finish(const DevPtrs &d, const StepConsts &k, uint32_t cap, cudaStream_t st) {
  k_writeback<<<grid_for(cap, 256), 256, 0, st>>>(d);
  k_prev_ranges<<<grid_for(k.n, 256), 256, 0, st>>>(d, k.n, cap);
  k_tool_partial<<<kToolBlocks, 256, 0, st>>>(d, k);
  k_tool_final<<<1, 32, 0, st>>>(d);
  k_integrate<<<grid_for(k.n, 256), 256, 0, st>>>(d, k);
  return 5;
}

void tds_launch_stage(const DevPtrs &d, uint32_t n, cudaStream_t st) {
  k_stage<<<grid_for(n, 256), 256, 0, st>>>(d, n);
}

const void *tds_pgs_kernel() { return (const void *)k_pgs; }
