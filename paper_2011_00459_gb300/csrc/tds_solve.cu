// tds_solve.cu -- the iterative PGS solve of the mesoscale MCP and the
// position update of the particle step (Algorithm 1).
//
// The MCP of the SPOOK stepper (section "Contacting rigid multibodies") is
// solved by projected Gauss-Seidel on the physical impulses, colour by
// colour: within a colour no two contacts share a particle, so all of them
// are updated in parallel and the result equals sequential Gauss-Seidel in
// colour-major order. One persistent, co-resident kernel runs the whole
// solve, each CTA waiting between colours only for the CTAs whose particles
// overlap its own (or, as an option, at a grid barrier): first
// v = M^-1 (p + G^T lambda_0) from the warm-start impulses, then the sweeps,
// with residual checks where the tolerance asks for them. Per contact and
// sweep: the normal row (clamped at -f_c), the 2-D tangent rows projected on
// the Coulomb disk mu |Lambda_n|, the 3 rolling rows projected on the ball
// rbar mu_r |Lambda_n| (Eqs. signCoul1-3), each followed by
// v += M^-1 G^T dLambda. Particle velocities are read and written through L2
// (ld.global.cg / st.global.cg) because other SMs update them between colours.
#include "tds_internal.cuh"

namespace {

__device__ __forceinline__ bool is_dyn(uint32_t b) { return (b & TDS_STATIC) == 0u; }

__global__ void k_predict(DevPtrs d, StepConsts k) {
  if (step_failed(d)) return;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n; i += gridDim.x * blockDim.x) {
    float4 v = d.pv[2 * i];
    if (v.w == 0.0f) continue;  // dormant reserve slot (1/m = 0): no gravity
    v.x += k.dt * k.g[0];
    v.y += k.dt * k.g[1];
    v.z += k.dt * k.g[2];
    d.pv[2 * i] = v;
  }
}

struct Side {
  float3 v, w;
  float im, iI;
};

__device__ __forceinline__ Side load_side(const DevPtrs &d, uint32_t s) {
  float4 v, w;
  ld_state(d.pv + 2 * (size_t)s, v, w);
  return Side{f3(v), f3(w), v.w, w.w};
}
__device__ __forceinline__ void store_side(const DevPtrs &d, uint32_t s, const Side &x) {
  st_state(d.pv + 2 * (size_t)s, make_float4(x.v.x, x.v.y, x.v.z, x.im),
           make_float4(x.w.x, x.w.y, x.w.z, x.iI));
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

// Projections on the Coulomb disk / rolling ball of radius bound (a zero
// bound forces zero). All solver arithmetic below spells out its rounding
// (see the vector helpers): every launch shape of the solver computes the
// same bits.
__device__ __forceinline__ void disk(float &a, float &b, float bound) {
  const float m2 = __fmaf_rn(b, b, __fmul_rn(a, a));
  if (m2 > __fmul_rn(bound, bound)) {
    const float s = bound > 0.f ? __fmul_rn(bound, rsqrtf(m2)) : 0.f;
    a = __fmul_rn(a, s);
    b = __fmul_rn(b, s);
  }
}
__device__ __forceinline__ void ball(float3 &a, float bound) {
  const float m2 = dot(a, a);
  if (m2 > __fmul_rn(bound, bound)) a = (bound > 0.f ? __fmul_rn(bound, rsqrtf(m2)) : 0.f) * a;
}

// v += M^-1 G^T dLambda for each row group. A static side has zero inverse
// mass and inertia, so its (discarded) update is a no-op.
__device__ __forceinline__ void apply_normal(const Row &r, Side &A, Side &B, float dn) {
  const float3 P = dn * r.n;
  A.v = axpy(-A.im, P, A.v);
  B.v = axpy(B.im, P, B.v);
}
__device__ __forceinline__ void apply_tangent(const Row &r, Side &A, Side &B, float3 dt) {
  const float3 c = cross(r.n, dt);  // torque arms: +la n on a, -lb n on b
  A.v = axpy(-A.im, dt, A.v);
  A.w = axpy(-__fmul_rn(A.iI, r.la), c, A.w);
  B.v = axpy(B.im, dt, B.v);
  B.w = axpy(-__fmul_rn(B.iI, r.lb), c, B.w);
}
__device__ __forceinline__ void apply_rolling(Side &A, Side &B, float3 dr) {
  A.w = axpy(-A.iI, dr, A.w);
  B.w = axpy(B.iI, dr, B.w);
}
// v += M^-1 G^T (dn, dt(world), dr) on both sides.
__device__ __forceinline__ void apply(const Row &r, Side &A, Side &B, float dn, float3 dt, float3 dr) {
  apply_normal(r, A, B, dn);
  apply_tangent(r, A, B, dt);
  apply_rolling(A, B, dr);
}

// Relative velocity of the contact points:
// (v_b + w_b x (-lb n)) - (v_a + w_a x (la n)) = (v_b - v_a) - (lb w_b + la w_a) x n
__device__ __forceinline__ float3 slip(const Row &r, const Side &A, const Side &B) {
  return (B.v - A.v) - cross(axpy(r.la, A.w, r.lb * B.w), r.n);
}

// Diagonal entries of the three row groups: 1/m_a + 1/m_b + Sigma_n,
// 1/m_a + 1/m_b + la^2/I_a + lb^2/I_b + sigma_t, 1/I_a + 1/I_b + sigma_r.
__device__ __forceinline__ float diag_n(const Row &r, const Side &A, const Side &B) {
  return __fadd_rn(__fadd_rn(A.im, B.im), r.Sn);
}
__device__ __forceinline__ float diag_t(const Row &r, const Side &A, const Side &B, float sig_t) {
  const float rot = __fmaf_rn(__fmul_rn(r.lb, r.lb), B.iI, __fmul_rn(__fmul_rn(r.la, r.la), A.iI));
  return __fadd_rn(__fadd_rn(__fadd_rn(A.im, B.im), rot), sig_t);
}
__device__ __forceinline__ float diag_r(const Side &A, const Side &B, float sig_r) {
  return __fadd_rn(__fadd_rn(A.iI, B.iI), sig_r);
}

// One projected Gauss-Seidel update of one contact.
__device__ __forceinline__ void pgs_update(const Row &r, Side &A, Side &B, float4 &L0, float2 &L1,
                                           float sig_t, float sig_r) {
  // normal row
  const float iDn = __frcp_rn(diag_n(r, A, B));
  const float res = __fsub_rn(__fmaf_rn(r.Sn, L0.x, dot(r.n, B.v - A.v)), r.qn);
  const float ln = fmaxf(__fmaf_rn(-res, iDn, L0.x), -r.fc);
  apply_normal(r, A, B, __fsub_rn(ln, L0.x));
  L0.x = ln;
  // tangent rows (Coulomb disk)
  float3 t1, t2;
  onb(r.n, t1, t2);
  const float iDt = __frcp_rn(diag_t(r, A, B, sig_t));
  const float3 u = slip(r, A, B);
  float y1 = __fmaf_rn(-__fmaf_rn(sig_t, L0.y, dot(t1, u)), iDt, L0.y);
  float y2 = __fmaf_rn(-__fmaf_rn(sig_t, L0.z, dot(t2, u)), iDt, L0.z);
  disk(y1, y2, __fmul_rn(r.mu, fabsf(ln)));
  apply_tangent(r, A, B, axpy(__fsub_rn(y2, L0.z), t2, __fsub_rn(y1, L0.y) * t1));
  L0.y = y1;
  L0.z = y2;
  // rolling rows (ball)
  const float iDr = __frcp_rn(diag_r(A, B, sig_r));
  const float3 lr = make_float3(L0.w, L1.x, L1.y);
  float3 y = axpy(-iDr, axpy(sig_r, lr, B.w - A.w), lr);
  ball(y, __fmul_rn(r.rmu, fabsf(ln)));
  apply_rolling(A, B, y - lr);
  L0.w = y.x;
  L1.x = y.y;
  L1.y = y.z;
}

// Contribution of one contact to the natural-map residual (Jacobi pass).
__device__ __forceinline__ void resid_terms(const Row &r, const Side &A, const Side &B, float4 L0,
                                            float2 L1, float sig_t, float sig_r, double &num,
                                            double &den) {
  const float wn = __fsub_rn(__fmaf_rn(r.Sn, L0.x, dot(r.n, B.v - A.v)), r.qn);
  const float pn = fmaxf(__fmaf_rn(-wn, __frcp_rn(diag_n(r, A, B)), L0.x), -r.fc);
  float3 t1, t2;
  onb(r.n, t1, t2);
  const float iDt = __frcp_rn(diag_t(r, A, B, sig_t));
  const float3 u = slip(r, A, B);
  float y1 = __fmaf_rn(-__fmaf_rn(sig_t, L0.y, dot(t1, u)), iDt, L0.y);
  float y2 = __fmaf_rn(-__fmaf_rn(sig_t, L0.z, dot(t2, u)), iDt, L0.z);
  disk(y1, y2, __fmul_rn(r.mu, fabsf(L0.x)));
  const float3 lr = make_float3(L0.w, L1.x, L1.y);
  float3 y = axpy(-__frcp_rn(diag_r(A, B, sig_r)), axpy(sig_r, lr, B.w - A.w), lr);
  ball(y, __fmul_rn(r.rmu, fabsf(L0.x)));
  const float e0 = __fsub_rn(L0.x, pn), e1 = __fsub_rn(L0.y, y1), e2 = __fsub_rn(L0.z, y2);
  const float3 e3 = lr - y;
  const float l2 = __fmaf_rn(L0.z, L0.z, __fmaf_rn(L0.y, L0.y, __fmul_rn(L0.x, L0.x)));
  num += (double)__fadd_rn(__fmaf_rn(e2, e2, __fmaf_rn(e1, e1, __fmul_rn(e0, e0))), dot(e3, e3));
  den += (double)__fadd_rn(l2, dot(lr, lr));
}

// Per-scene stop state of the solver (a bit per scene in shared memory).
__device__ __forceinline__ bool scene_done(const uint32_t *done, uint32_t q) {
  return (done[q >> 5] >> (q & 31u)) & 1u;
}
// The residual r of scene q at sweep it: CTA 0 keeps it as the scene's latest
// (residual, sweeps); below the tolerance the scene is marked to stop, else it
// competes for the largest residual of the scenes still sweeping (r >= 0, so
// its bits order like the values).
__device__ __forceinline__ void record_scene(const DevPtrs &d, uint32_t q, float r, float tol, uint32_t it,
                                             uint32_t *done_new, uint32_t *rmax) {
  if (blockIdx.x == 0) {
    d.scene_res[q] = r;
    d.scene_iters[q] = it;
  }
  if (tol > 0.f && r <= tol) atomicOr(done_new + (q >> 5), 1u << (q & 31u));
  else atomicMax(rmax, __float_as_uint(r));
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
  int sync;  // between colours: 0 grid barrier, 1 neighbour synchronisation
  uint32_t n;  // particle slots
};

// ---------------------------------------------------------------------------
// Staging of the contact rows and impulses with bulk copies (TMA)
// ---------------------------------------------------------------------------
// CTA shapes compiled: (threads, contacts per thread, co-resident CTAs per
// SM the register budget is sized for); launch configurations choose one by
// index. In every shape the last warp stages the waves and the others solve
// (a wave is (threads - 32) x contacts per thread, see pgs_wave). The first
// is the default, measured fastest on the 1M bed: two 416-thread CTAs per SM
// (384 solving threads each, one contact per thread). Each colour phase is a
// latency chain of which a thread's serial updates are a large part, and the
// second CTA keeps the SM busy while the first waits.
constexpr int kShapes[][3] = {{416, 1, 2}, {768, 1, 1}, {512, 2, 1}, {640, 2, 1}, {512, 3, 1}, {256, 1, 3}};
constexpr int kNumShapes = 6;
constexpr int kStages = 2;                           // waves in flight
constexpr uint32_t kFirstCheck = 5;                  // first residual check in adaptive mode
constexpr uint32_t kResSum = 256;                    // residual: threads adding up a large scene's chunks
constexpr uint32_t kWarpChunks = 1024;               // residual: scenes with at most this many chunks
                                                     // are added by one warp, larger ones by the CTA
// per contact: ab 8 | (n, la) 16 | (lb, q_n, Sigma_n, f_c) 16 | (mu, rbar mu_r) 8 |
//              impulses (n, t1, t2, r.x) 16 | (r.y, r.z) 8
constexpr size_t kRowBytes = 72;
constexpr size_t kOffAb = 0, kOffRn = 8, kOffRq = 24, kOffRm = 40, kOffLa = 48, kOffLb = 64;  // x wave size
__host__ __device__ constexpr size_t stage_bytes(int wave) { return (size_t)wave * kRowBytes; }
__host__ __device__ constexpr size_t pgs_smem(int wave) { return kStages * stage_bytes(wave); }
// The last warp of a CTA stages the waves (bulk copies take the issuing
// thread a long time each: on a computing warp they would hold up every
// wave's barrier); the other warps solve, one wave = their threads x the
// contacts per thread.
__host__ __device__ constexpr int pgs_wave(int threads, int per_thread) { return (threads - 32) * per_thread; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait of one thread for a phase of a stage barrier; false (error
// latched) when it has waited longer than limit_ns, or (if early) at once
// when the step has already failed. The wait for the copies still in flight
// before a CTA exits is not early: it gives those copies their full time.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, int32_t *err,
                                          unsigned long long limit_ns, bool early = true) {
  unsigned long long t0 = 0;
  for (unsigned k = 0;; ++k) {
    if (mbar_test(bar, parity)) return true;
    if (k == 0) t0 = global_ns();
    if ((k & 15u) == 15u) {
      if (early && *(volatile int32_t *)err != 0) return false;  // the step has failed already
      if (global_ns() - t0 > limit_ns) {
        latch_error(err, DEV_ERR_BARRIER);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Segments: colour c has two, 2c (its particle-pair bucket) and 2c + 1 (its
// static bucket). Each CTA takes the same share [lo, hi) of both, starting at
// a multiple of 4 contacts, so its work in every colour lies in the same
// stretch of slot order (buckets keep the owner order).
__device__ __forceinline__ void seg_chunk(const DevPtrs &d, uint32_t g, uint32_t &lo, uint32_t &hi) {
  const uint32_t s = d.bstart[g], e = d.bend[g];
  uint32_t q = (e - s + gridDim.x - 1) / gridDim.x;
  q = (q + 3u) & ~3u;
  lo = min(s + blockIdx.x * q, e);
  hi = min(lo + q, e);
}

// One wave of a colour: up to W contacts of this CTA's pair chunk
// [lo1, hi1), then of its static chunk [lo2, hi2). The pair part n1 sits at
// stage entries [0, n1), the static part n2 at [n1e, n1e + n2) with n1e = n1
// rounded up to even (8-byte fields are copied in 16-byte pairs); n1e + n2 <=
// W. Waves of a colour: the pair chunk in W pieces, the last one
// topped up with static contacts, then the rest of the static chunk.
struct WaveDesc {
  uint32_t a1, n1, n1e, a2, n2;
};

__device__ __forceinline__ uint32_t waves_of(uint32_t L1, uint32_t L2, uint32_t W) {
  const uint32_t W1 = (L1 + W - 1) / W;
  uint32_t first2 = 0;  // static contacts in the last pair wave
  if (W1 > 0) {
    const uint32_t n1 = L1 - (W1 - 1) * W;
    first2 = min(L2, W - ((n1 + 1u) & ~1u));
  }
  return W1 + (L2 - first2 + W - 1) / W;
}

__device__ __forceinline__ WaveDesc wave_desc(uint32_t lo1, uint32_t hi1, uint32_t lo2, uint32_t hi2, uint32_t w,
                                              uint32_t W) {
  const uint32_t L1 = hi1 - lo1, L2 = hi2 - lo2;
  const uint32_t W1 = (L1 + W - 1) / W;
  WaveDesc q{0, 0, 0, lo2, 0};
  uint32_t first2 = 0;
  if (W1 > 0) {
    const uint32_t n1 = L1 - (W1 - 1) * W;
    first2 = min(L2, W - ((n1 + 1u) & ~1u));
  }
  if (w < W1) {
    q.a1 = lo1 + w * W;
    q.n1 = min(W, L1 - w * W);
    q.n1e = (q.n1 + 1u) & ~1u;
    if (w == W1 - 1) q.n2 = first2;
  } else {
    const uint32_t done = first2 + (w - W1) * W;
    q.a2 = lo2 + done;
    q.n2 = min(W, L2 - done);
  }
  return q;
}

// Walks the (sweep, colour, wave) sequence of this CTA's staged waves.
struct WaveSeq {
  uint32_t sweep, col, w;
  __device__ bool valid(uint32_t max_iters) const { return sweep < max_iters; }
  // moves to the next wave, skipping colours without waves for this CTA
  __device__ void advance(const uint32_t *nw, uint32_t ncol, uint32_t max_iters) {
    ++w;
    while (sweep < max_iters && w >= nw[col]) {
      w = 0;
      if (++col >= ncol) { col = 0; ++sweep; }
    }
  }
};

__device__ __forceinline__ void stage_range(const DevPtrs &d, uint32_t p0, uint32_t cnt, uint32_t at,
                                            unsigned char *stage, unsigned long long *bar, uint32_t W) {
  const uint32_t cnt2 = (cnt + 1u) & ~1u;  // 8-byte fields copied in pairs (16-byte multiples)
  bulk_g2s(stage + kOffAb * W + 8u * at, d.p_ab + p0, 8u * cnt2, bar);
  bulk_g2s(stage + kOffRn * W + 16u * at, d.p_rn + p0, 16u * cnt, bar);
  bulk_g2s(stage + kOffRq * W + 16u * at, d.p_rq + p0, 16u * cnt, bar);
  bulk_g2s(stage + kOffRm * W + 8u * at, d.p_rm + p0, 8u * cnt2, bar);
  bulk_g2s(stage + kOffLa * W + 16u * at, d.p_la + p0, 16u * cnt, bar);
  bulk_g2s(stage + kOffLb * W + 8u * at, d.p_lb + p0, 8u * cnt2, bar);
}

__device__ __forceinline__ uint32_t range_bytes(uint32_t cnt) {
  return cnt ? 3u * 16u * cnt + 3u * 8u * ((cnt + 1u) & ~1u) : 0u;
}

__device__ __forceinline__ void issue_wave(const DevPtrs &d, const WaveSeq &q, const uint32_t *lo,
                                           const uint32_t *hi, unsigned char *stage,
                                           unsigned long long *bar, uint32_t W) {
  const WaveDesc w = wave_desc(lo[2 * q.col], hi[2 * q.col], lo[2 * q.col + 1], hi[2 * q.col + 1], q.w, W);
  mbar_expect_tx(bar, range_bytes(w.n1) + range_bytes(w.n2));
  if (w.n1) stage_range(d, w.a1, w.n1, 0, stage, bar, W);
  if (w.n2) stage_range(d, w.a2, w.n2, w.n1e, stage, bar, W);
}

// Neighbour synchronisation. Every CTA touches particles only inside its slot
// range [rng_lo, rng_hi] (both sides of all its contacts, all colours); its
// neighbours are the CTAs whose ranges overlap it (a symmetric relation).
// Before colour phase t a CTA waits until each neighbour has published phase
// t - 1; after its own stores of phase t it publishes t. Every write to a
// particle before phase t then comes from a neighbour that has finished it,
// and no neighbour can still be reading a particle this CTA writes, so the
// result equals the grid-barrier order bit for bit. The least advanced CTA
// never waits, so the scheme cannot deadlock. The threads poll the
// neighbours between them; waits are bounded like grid_barrier.
__device__ __forceinline__ bool neighbour_wait(const DevPtrs &d, uint32_t jlo, uint32_t jhi, uint32_t target,
                                               int *s_fail) {
  // thread t polls neighbours jlo + t, jlo + t + blockDim.x, ... (a range can
  // be wider than the CTA when few contacts of a colour spread over the bed)
  for (uint32_t j = jlo + threadIdx.x; j <= jhi; j += blockDim.x) {
    if (j == blockIdx.x) continue;
    unsigned long long t0 = 0;
    for (unsigned spins = 0;; ++spins) {
      uint32_t cur;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(d.prog + kProgStride * j) : "memory");
      if ((int32_t)(cur - target) >= 0) break;
      if ((spins & 31u) == 31u) {
        if (*(volatile int32_t *)d.err != 0) { *s_fail = 1; break; }
        unsigned long long t = global_ns();
        if (t0 == 0) t0 = t;
        else if (t - t0 > d.wait_ns) {
          latch_error(d.err, DEV_ERR_BARRIER);
          *s_fail = 1;
          break;
        }
      }
    }
    if (*(volatile int *)s_fail) break;
  }
  __syncthreads();
  return *s_fail == 0;
}

// Publishes phase t of this CTA; the caller has passed a __syncthreads after
// the phase's stores (the release is cumulative over them).
__device__ __forceinline__ void publish(const DevPtrs &d, uint32_t t) {
  if (threadIdx.x == 0)
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(d.prog + kProgStride * blockIdx.x), "r"(t)
                 : "memory");
}

// The persistent solver: kMinBlocks co-resident CTAs per SM; between colours
// either a grid barrier or neighbour synchronisation. The rows and impulses
// of each wave (up to kWave contacts of one segment) are staged in shared
// memory by bulk copies that the CTA's last warp issues ahead, so they stream
// from HBM while earlier colours are solved and synchronised; each solving
// thread then gathers both sides of its kPerThread contacts (through L2)
// before solving any of them (contacts of one colour touch disjoint
// particles).
template <int kPgsThreads, int kPerThread, int kMinBlocks>
__global__ void __launch_bounds__(kPgsThreads, kMinBlocks) k_pgs(DevPtrs d, SolveArgs a) {
  constexpr uint32_t kCompute = kPgsThreads - 32;      // solving threads; the last warp stages
  constexpr uint32_t kProducer = kCompute;             // the staging thread (lane 0 of the last warp)
  constexpr uint32_t kWave = pgs_wave(kPgsThreads, kPerThread);  // contacts per wave
  constexpr size_t kStageBytes = stage_bytes(kWave);
  if (step_failed(d)) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned long long full[kStages];
  __shared__ uint32_t s_lo[2 * TDS_MAX_COLOURS], s_hi[2 * TDS_MAX_COLOURS], s_nw[TDS_MAX_COLOURS];
  __shared__ double s_rn[kResSum], s_rd[kResSum];
  static_assert(kPgsThreads >= (int)kResSum, "the residual sum needs kResSum threads");
  __shared__ uint32_t s_mn[kPgsThreads / 32], s_mx[kPgsThreads / 32];
  __shared__ int s_flag, s_fail, s_gaveup;
  __shared__ uint32_t s_waves, s_jlo, s_jhi;
  __shared__ uint32_t s_done[TDS_MAX_SCENES / 32], s_done_new[TDS_MAX_SCENES / 32];
  __shared__ uint32_t s_rmax, s_ndone, s_ndone_check;
  __shared__ unsigned long long s_acc[2];
  const uint32_t ncol = min(d.ctr[CTR_NCOL], (uint32_t)TDS_MAX_COLOURS);
  const uint32_t nseg = 2 * ncol;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t stride = gridDim.x * blockDim.x;
  if (threadIdx.x == 0) {
    s_waves = 0;
    s_fail = 0;
    s_gaveup = 0;  // a wait for a staged wave gave up
    s_jlo = s_jhi = blockIdx.x;
    s_ndone = 0;
    s_acc[0] = s_acc[1] = 0ull;
  }
  for (uint32_t w = threadIdx.x; w < TDS_MAX_SCENES / 32; w += blockDim.x) s_done[w] = 0u;
  __syncthreads();
  for (uint32_t g = threadIdx.x; g < nseg; g += blockDim.x) seg_chunk(d, g, s_lo[g], s_hi[g]);
  __syncthreads();
  for (uint32_t c = threadIdx.x; c < ncol; c += blockDim.x) {
    s_nw[c] = waves_of(s_hi[2 * c] - s_lo[2 * c], s_hi[2 * c + 1] - s_lo[2 * c + 1], kWave);
    atomicAdd(&s_waves, s_nw[c]);
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < kStages; ++k) mbar_init(&full[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint32_t waves_per_sweep = s_waves;
  uint32_t gen = 0;  // grid barriers passed

  if (a.sync) {  // this CTA's touched slot range, then its neighbours
    uint32_t mn = 0xFFFFFFFFu, mx = 0u;
    for (uint32_t g = 0; g < nseg; ++g)
      for (uint32_t p = s_lo[g] + threadIdx.x; p < s_hi[g]; p += blockDim.x) {
        const uint2 ab = __ldcg(d.p_ab + p);
        if (ab.x == 0xFFFFFFFFu) continue;  // padding slot
        mn = min(mn, ab.x);
        mx = max(mx, ab.x);
        if (is_dyn(ab.y)) {
          mn = min(mn, ab.y);
          mx = max(mx, ab.y);
        }
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
      s_mn[threadIdx.x >> 5] = mn;
      s_mx[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kPgsThreads / 32; ++w) {
        mn = min(mn, s_mn[w]);
        mx = max(mx, s_mx[w]);
      }
      __stcg(d.rng + 2 * blockIdx.x, mn);
      __stcg(d.rng + 2 * blockIdx.x + 1, mx);
      s_mn[0] = mn;
      s_mx[0] = mx;
    }
    if (!grid_barrier(d.bar, d.err, gen, d.wait_ns)) return;
    const uint32_t lo = s_mn[0], hi = s_mx[0];
    for (uint32_t j = threadIdx.x; j < gridDim.x; j += blockDim.x) {
      const uint32_t jl = __ldcg(d.rng + 2 * j), jh = __ldcg(d.rng + 2 * j + 1);
      if (lo <= hi && jl <= jh && max(lo, jl) <= min(hi, jh)) {
        atomicMin(&s_jlo, j);
        atomicMax(&s_jhi, j);
      }
    }
    __syncthreads();
  }
  const uint32_t jlo = s_jlo, jhi = s_jhi;
  // staged impulses of a wave were written one sweep earlier by this CTA, so
  // never run further ahead than one sweep's worth of waves
  const uint32_t ahead = min((uint32_t)kStages, waves_per_sweep);

  // v = M^-1 (p + G^T lambda_0), colour by colour (no conflicts inside one)
  if (a.apply_warm) {
    for (uint32_t col = 0; col < ncol; ++col) {
      for (int part = 0; part < 2; ++part) {
        const uint32_t s = d.bstart[2 * col + part], e = d.bend[2 * col + part];
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
      }
      if (!grid_barrier(d.bar, d.err, gen, d.wait_ns)) return;
    }
  }

  // producer (thread kProducer): the next wave to stage
  uint32_t issued = 0, consumed = 0;
  WaveSeq prod{0, 0, 0xFFFFFFFFu};
  if (waves_per_sweep > 0 && a.max_iters > 0) {
    prod.advance(s_nw, ncol, a.max_iters);  // first wave
    if (threadIdx.x == kProducer)
      for (uint32_t k = 0; k < ahead && prod.valid(a.max_iters); ++k) {
        issue_wave(d, prod, s_lo, s_hi, smem + (size_t)(issued % kStages) * kStageBytes,
                   &full[issued % kStages], kWave);
        ++issued;
        prod.advance(s_nw, ncol, a.max_iters);
      }
  }

  bool ok = true;
  uint32_t it = 0;
  float resid = -1.f;
  // residual checks: every `every` sweeps, or (every == 0) where the decay
  // seen so far says the tolerance will be met (see below)
  __shared__ uint32_t s_next;
  uint32_t next_check = a.every ? a.every : kFirstCheck;
  float prev_res = -1.f;
  uint32_t prev_it = 0;
  while (ok && it < a.max_iters) {
    for (uint32_t col = 0; col < ncol; ++col) {
      const uint32_t phase = it * ncol + col + 1u;
      const bool busy = s_nw[col] > 0;
      if (a.sync && busy && !neighbour_wait(d, jlo, jhi, phase - 1u, &s_fail)) { ok = false; break; }
      for (uint32_t w = 0; w < s_nw[col]; ++w) {
        const uint32_t st = consumed % kStages;
        unsigned char *stage = smem + (size_t)st * kStageBytes;
        // a wait for this CTA's own bulk copies (which complete in
        // microseconds): the fixed limit, not the limit on waits for others
        // A wait that gives up (the error is latched) skips this wave, and no
        // thread leaves the loop here: every CTA leaves it together at the
        // next residual check, whose grid barrier sees the error. The CTA
        // stages no wave after it; particle indices read from a stage are
        // checked against the particle count all the same.
        const bool staged =
            threadIdx.x < kCompute && mbar_wait(&full[st], (consumed / kStages) & 1u, d.err, TDS_BARRIER_NS);
        if (!staged && threadIdx.x < kCompute) s_gaveup = 1;  // read by the staging thread after the barrier
        const uint2 *sab = reinterpret_cast<const uint2 *>(stage + kOffAb * kWave);
        const float4 *srn = reinterpret_cast<const float4 *>(stage + kOffRn * kWave);
        const float4 *srq = reinterpret_cast<const float4 *>(stage + kOffRq * kWave);
        const float2 *srm = reinterpret_cast<const float2 *>(stage + kOffRm * kWave);
        const float4 *sla = reinterpret_cast<const float4 *>(stage + kOffLa * kWave);
        const float2 *slb = reinterpret_cast<const float2 *>(stage + kOffLb * kWave);
        const WaveDesc q = wave_desc(s_lo[2 * col], s_hi[2 * col], s_lo[2 * col + 1], s_hi[2 * col + 1], w, kWave);
        Side A[kPerThread], B[kPerThread];
        uint32_t gp[kPerThread];  // colour-order index of each staged contact (or ~0)
        uint32_t qs[kPerThread];  // its scene, once some scene of a batch has stopped
        const bool skip_done = s_ndone != 0u;
        // gathers of every contact of this thread first (disjoint particles)
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
          const uint32_t li = j * kCompute + threadIdx.x;
          gp[j] = !staged ? ~0u
                  : li < q.n1 ? q.a1 + li : (li >= q.n1e && li < q.n1e + q.n2 ? q.a2 + (li - q.n1e) : ~0u);
          if (gp[j] != ~0u) {
            const uint2 ab = sab[li];
            if (ab.x < a.n && (!is_dyn(ab.y) || ab.y < a.n)) {  // not a padding slot (all ones)
              if (skip_done) qs[j] = __ldcg(d.sid + ab.x);
              A[j] = load_side(d, ab.x);
              if (is_dyn(ab.y)) B[j] = load_side(d, ab.y);
              else B[j] = Side{f3(d.p_sv[gp[j]]), f3(d.p_sw[gp[j]]), 0.f, 0.f};
            }
          }
        }
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
          const uint32_t li = j * kCompute + threadIdx.x;
          if (gp[j] != ~0u) {
            Row r;
            r.ab = sab[li];
            if (r.ab.x >= a.n || (is_dyn(r.ab.y) && r.ab.y >= a.n)) continue;  // padding slot
            if (skip_done && scene_done(s_done, qs[j])) continue;  // its scene met the tolerance
            const float4 rn = srn[li], rq = srq[li];
            const float2 rm = srm[li];
            r.n = f3(rn); r.la = rn.w;
            r.lb = rq.x; r.qn = rq.y; r.Sn = rq.z; r.fc = rq.w;
            r.mu = rm.x; r.rmu = rm.y;
            r.dyn = is_dyn(r.ab.y);
            float4 L0 = sla[li];
            float2 L1 = slb[li];
            pgs_update(r, A[j], B[j], L0, L1, a.sig_t, a.sig_r);
            store_side(d, r.ab.x, A[j]);
            if (r.dyn) store_side(d, r.ab.y, B[j]);
            d.p_la[gp[j]] = L0;
            d.p_lb[gp[j]] = L1;
          }
        }
        // impulses written above are read back by bulk copies one sweep later
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncthreads();  // the stage is free again
        ++consumed;
        // (no more waves once a wait of this CTA has given up: its stage may
        // still have a copy landing in it)
        if (threadIdx.x == kProducer && prod.valid(a.max_iters) && !*(volatile int *)&s_gaveup) {
          issue_wave(d, prod, s_lo, s_hi, smem + (size_t)(issued % kStages) * kStageBytes,
                     &full[issued % kStages], kWave);
          ++issued;
          prod.advance(s_nw, ncol, a.max_iters);
        }
      }
      if (!ok) break;
      if (a.sync) publish(d, phase);
      else if (!grid_barrier(d.bar, d.err, gen, d.wait_ns)) { ok = false; break; }
    }
    if (!ok) break;
    ++it;
    if (it == a.max_iters || (a.tol > 0.f && it == next_check)) {
      // the residual reads every contact: all colours of this sweep first
      if (a.sync && !grid_barrier(d.bar, d.err, gen, d.wait_ns)) { ok = false; break; }
      // Every scene has its own residual, summed in an order that neither the
      // launch shape nor the other scenes of a batch change: its chunks (its
      // contacts of one bucket, at most TDS_RES_CHUNK of them, consecutive in
      // the colour order) are each added by one warp (lane l takes l, l + 32,
      // ..., then a fixed shuffle tree); then every CTA adds each scene's
      // chunk sums the same way, so all CTAs take the same stop decisions
      // from the same values. A scene that met the tolerance stops sweeping
      // and keeps the residual of that check.
      const uint32_t nchunk = d.ctr[CTR_NCHUNK];
      const uint32_t lane = threadIdx.x & 31u;
      for (uint32_t ch = tid >> 5; ch < nchunk; ch += stride >> 5) {
        const uint4 cd = __ldcg(d.chunk + ch);
        if (scene_done(s_done, cd.z)) continue;
        double cn = 0.0, cdn = 0.0;
        for (uint32_t q = lane; q < cd.y; q += 32u) {
          const uint32_t p = cd.x + q;
          Row r = load_row(d, p);
          Side A, B;
          load_pair(d, r, A, B);
          resid_terms(r, A, B, __ldcg(d.p_la + p), __ldcg(d.p_lb + p), a.sig_t, a.sig_r, cn, cdn);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          cn += __shfl_down_sync(0xffffffffu, cn, o);
          cdn += __shfl_down_sync(0xffffffffu, cdn, o);
        }
        if (lane == 0) {
          __stcg(d.dres + 2 * ch, cn);
          __stcg(d.dres + 2 * ch + 1, cdn);
        }
      }
      if (!grid_barrier(d.bar, d.err, gen, d.wait_ns)) { ok = false; break; }
      const uint32_t S = d.nscenes;
      for (uint32_t w = threadIdx.x; w < (S + 31u) / 32u; w += blockDim.x) s_done_new[w] = 0u;
      if (threadIdx.x == 0) s_rmax = 0u;
      __syncthreads();
      // scenes with many chunks: the whole CTA adds them (fixed strides, fixed tree)
      for (uint32_t q = 0; q < S; ++q) {
        const uint32_t c0 = __ldcg(d.scq_chunk + (size_t)q * TDS_NBUCKETS);
        const uint32_t c1 = __ldcg(d.scq_chunk + (size_t)(q + 1) * TDS_NBUCKETS);
        if (c1 - c0 <= kWarpChunks || scene_done(s_done, q)) continue;
        if (threadIdx.x < kResSum) {
          double n0 = 0.0, n1 = 0.0, d0 = 0.0, d1 = 0.0;
          uint32_t ch = c0 + threadIdx.x;
          for (; ch + kResSum < c1; ch += 2u * kResSum) {
            const double2 u = __ldcg(reinterpret_cast<const double2 *>(d.dres) + ch);
            const double2 v = __ldcg(reinterpret_cast<const double2 *>(d.dres) + ch + kResSum);
            n0 += u.x; d0 += u.y;
            n1 += v.x; d1 += v.y;
          }
          if (ch < c1) {
            const double2 u = __ldcg(reinterpret_cast<const double2 *>(d.dres) + ch);
            n0 += u.x; d0 += u.y;
          }
          s_rn[threadIdx.x] = n0 + n1;
          s_rd[threadIdx.x] = d0 + d1;
        }
        __syncthreads();
        for (uint32_t h = kResSum / 2u; h > 0u; h >>= 1) {
          if (threadIdx.x < h) {
            s_rn[threadIdx.x] += s_rn[threadIdx.x + h];
            s_rd[threadIdx.x] += s_rd[threadIdx.x + h];
          }
          __syncthreads();
        }
        if (threadIdx.x == 0)
          record_scene(d, q, (float)(sqrt(s_rn[0]) / fmax(sqrt(s_rd[0]), 1e-12)), a.tol, it, s_done_new, &s_rmax);
        __syncthreads();
      }
      // the other scenes: one warp each (lane strides, fixed shuffle tree)
      for (uint32_t q = threadIdx.x >> 5; q < S; q += blockDim.x >> 5) {
        const uint32_t c0 = __ldcg(d.scq_chunk + (size_t)q * TDS_NBUCKETS);
        const uint32_t c1 = __ldcg(d.scq_chunk + (size_t)(q + 1) * TDS_NBUCKETS);
        if (c1 - c0 > kWarpChunks || scene_done(s_done, q)) continue;
        double tn = 0.0, td = 0.0;
        for (uint32_t ch = c0 + lane; ch < c1; ch += 32u) {
          const double2 u = __ldcg(reinterpret_cast<const double2 *>(d.dres) + ch);
          tn += u.x;
          td += u.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          tn += __shfl_down_sync(0xffffffffu, tn, o);
          td += __shfl_down_sync(0xffffffffu, td, o);
        }
        if (lane == 0) record_scene(d, q, (float)(sqrt(tn) / fmax(sqrt(td), 1e-12)), a.tol, it, s_done_new, &s_rmax);
      }
      __syncthreads();
      if (threadIdx.x == 0) s_ndone_check = 0u;
      __syncthreads();
      for (uint32_t w = threadIdx.x; w < (S + 31u) / 32u; w += blockDim.x) {
        s_done[w] |= s_done_new[w];
        atomicAdd(&s_ndone_check, (uint32_t)__popc(s_done[w]));
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        s_ndone = s_ndone_check;
        // the largest residual of the scenes still sweeping (0 when all stopped)
        resid = __uint_as_float(s_rmax);
        s_flag = a.tol > 0.f && s_ndone == S;
        // next check: a fixed period, or the sweep where the geometric decay
        // of that residual between the last two checks reaches the tolerance
        // (at least 2 and at most 64 sweeps on); every CTA computes the same
        // value from the same residuals
        uint32_t gap = a.every;
        if (a.every == 0) {
          gap = kFirstCheck;
          if (prev_res > 0.f && resid < prev_res && resid > a.tol) {
            const double rate = log((double)resid / (double)prev_res) / (double)(it - prev_it);
            const double need = ceil(log((double)a.tol / (double)resid) / rate);
            gap = (uint32_t)fmin(64.0, fmax(2.0, need));
          }
          prev_res = resid;
          prev_it = it;
        }
        s_next = it + gap;
      }
      __syncthreads();
      next_check = s_next;
      if (s_flag) break;
    }
  }
  // drain the waves still in flight before the CTA exits (bulk copies of this
  // CTA's own: a fixed, generous limit, whatever the limit on waits for others)
  if (threadIdx.x == kProducer)
    for (uint32_t q = consumed; q < issued; ++q)
      if (!mbar_wait(&full[q % kStages], (q / kStages) & 1u, d.err, TDS_BARRIER_NS, false)) break;
  const bool all_ok = __syncthreads_and(ok) != 0;  // every thread of the CTA reaches this point
  if (blockIdx.x == 0 && all_ok) {
    // statistics: the sweeps done (the most any scene did), the largest final
    // residual, and per scene its sweeps x its contacts (the solver's work)
    __syncthreads();
    const uint32_t S = d.nscenes;
    if (it == 0u)
      for (uint32_t q = threadIdx.x; q < S; q += blockDim.x) {
        d.scene_iters[q] = 0u;
        d.scene_res[q] = -1.f;
      }
    __syncthreads();
    if (threadIdx.x == 0) s_rmax = 0u;
    __syncthreads();
    unsigned long long pp = 0ull, sc = 0ull;
    for (uint32_t q = threadIdx.x; q < S; q += blockDim.x) {
      const unsigned long long iq = d.scene_iters[q];
      for (uint32_t b = 0; b < TDS_NBUCKETS; ++b) {
        const unsigned long long c = d.scq_cnt[(size_t)q * TDS_NBUCKETS + b];
        if (b & 1u) sc += iq * c;
        else pp += iq * c;
      }
      const float r = d.scene_res[q];
      if (r > 0.f) atomicMax(&s_rmax, __float_as_uint(r));
    }
    if (pp) atomicAdd(&s_acc[0], pp);
    if (sc) atomicAdd(&s_acc[1], sc);
    __syncthreads();
    if (threadIdx.x == 0) {
      d.ctr[CTR_ITERS] = it;
      d.fscal[FS_RESID] = it == 0u ? -1.f : __uint_as_float(s_rmax);
      d.acc[ACC_SWEEP_PP] += s_acc[0];
      d.acc[ACC_SWEEP_ST] += s_acc[1];
      d.acc[ACC_CONTACTS] += d.ctr[CTR_NC];
      d.acc[ACC_STEPS] += 1;
    }
  }
}

// Impact stage (the Newton impact law): a rigid velocity-level solve on the
// predicted velocities v* before the main solve. Pass 0 classifies every
// contact by its approach speed at the start of the step, -G_n v_n (G_n v* for
// a particle pair; G_n v* + h n.g against a static surface, which does not
// fall), sets the normal target e * approach for impacts and 0 otherwise, and
// zeroes the stage's impulses; with no impact the kernel stops there. Then
// `iters` colour sweeps of the main solve's update on rows with no compliance
// (Sigma_n = 0), that target as q_n and no cohesion; finally every contact's
// q_n takes the post-impact normal velocity: q_n += Upsilon (G_n v+ - G_n v*).
struct ImpactArgs {
  float e, vimp, h, g[3], ups, sig_t, sig_r;
  uint32_t iters;
};

__global__ void __launch_bounds__(512) k_impact(DevPtrs d, ImpactArgs a) {
  if (step_failed(d)) return;
  __shared__ uint32_t s_count;
  const uint32_t ncol = min(d.ctr[CTR_NCOL], (uint32_t)TDS_MAX_COLOURS);
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  uint32_t gen = 0;
  if (threadIdx.x == 0) s_count = 0;
  __syncthreads();
  uint32_t mine = 0;
  for (uint32_t col = 0; col < ncol; ++col)
    for (int part = 0; part < 2; ++part)
      for (uint32_t p = d.bstart[2 * col + part] + tid; p < d.bend[2 * col + part]; p += stride) {
        const Row r = load_row(d, p);
        Side A, B;
        load_pair(d, r, A, B);
        const float gv = dot(r.n, B.v - A.v);
        const float gvn = r.dyn ? gv : gv + a.h * (r.n.x * a.g[0] + r.n.y * a.g[1] + r.n.z * a.g[2]);
        const bool hit = -gvn > a.vimp;
        mine += hit;
        d.p_il[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        d.p_il2[p] = make_float4(0.f, 0.f, gv, hit ? a.e * -gvn : 0.f);
      }
  if (mine) atomicAdd(&s_count, mine);
  __syncthreads();
  if (threadIdx.x == 0 && s_count) atomicAdd(d.ctr + CTR_IMPACTS, s_count);
  if (!grid_barrier(d.bar, d.err, gen, d.wait_ns)) return;
  if (*(volatile uint32_t *)(d.ctr + CTR_IMPACTS) == 0) return;  // the same value in every CTA
  for (uint32_t it = 0; it < a.iters; ++it)
    for (uint32_t col = 0; col < ncol; ++col) {
      for (int part = 0; part < 2; ++part)
        for (uint32_t p = d.bstart[2 * col + part] + tid; p < d.bend[2 * col + part]; p += stride) {
          Row r = load_row(d, p);
          const float4 t = d.p_il2[p];
          r.Sn = 0.f;
          r.fc = 0.f;
          r.qn = t.w;
          float4 L0 = d.p_il[p];
          float2 L1 = make_float2(t.x, t.y);
          Side A, B;
          load_pair(d, r, A, B);
          pgs_update(r, A, B, L0, L1, a.sig_t, a.sig_r);
          store_side(d, r.ab.x, A);
          if (r.dyn) store_side(d, r.ab.y, B);
          d.p_il[p] = L0;
          d.p_il2[p] = make_float4(L1.x, L1.y, t.z, t.w);
        }
      if (!grid_barrier(d.bar, d.err, gen, d.wait_ns)) return;
    }
  for (uint32_t col = 0; col < ncol; ++col)
    for (int part = 0; part < 2; ++part)
      for (uint32_t p = d.bstart[2 * col + part] + tid; p < d.bend[2 * col + part]; p += stride) {
        const Row r = load_row(d, p);
        Side A, B;
        load_pair(d, r, A, B);
        d.p_rq[p].y = r.qn + a.ups * (dot(r.n, B.v - A.v) - d.p_il2[p].z);
      }
}

// Colour order -> owner order warm-start memory: (key's other side,
// impulses with the tangent in world coordinates); per particle id the range
// of its owned contacts.
__global__ void k_writeback(DevPtrs d) {
  if (step_failed(d)) return;
  const uint32_t np = d.ctr[CTR_PADDED];
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    uint32_t c = d.order[p];
    if (c == 0xFFFFFFFFu) continue;  // padding slot
    float4 L0 = d.p_la[p];
    float2 L1 = d.p_lb[p];
    float3 n = f3(d.p_rn[p]), t1, t2;
    onb(n, t1, t2);
    float3 tw = L0.y * t1 + L0.z * t2;
    d.prev_other[1][c] = (uint32_t)(d.c_key[c] & 0xFFFFFFFFull);
    d.prev_l0[1][c] = make_float4(L0.x, tw.x, tw.y, tw.z);
    d.prev_l1[1][c] = make_float4(L0.w, L1.x, L1.y, __uint_as_float((uint32_t)d.colour[c]));  // + its colour
    if (d.targ) {  // training targets of the learned warm start (final impulses in the slip frame)
      const float4 sw = d.sdirw[c];
      const float3 s = f3(sw);
      d.targ[3 * (size_t)c] = L0.x / sw.w;
      d.targ[3 * (size_t)c + 1] = dot(tw, s) / sw.w;
      d.targ[3 * (size_t)c + 2] = dot(tw, cross(n, s)) / sw.w;
    }
  }
}

__global__ void k_prev_ranges(DevPtrs d, uint32_t n, uint32_t cap) {
  if (step_failed(d)) return;
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
  if (step_failed(d)) return;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n; i += gridDim.x * blockDim.x) {
    float4 p = d.pos[i], v = d.pv[2 * i], w = d.pv[2 * i + 1];
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
  if (step_failed(d)) return;
  __shared__ double sh[8];
  const uint32_t np = d.ctr[CTR_PADDED];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    if (d.order[p] == 0xFFFFFFFFu) continue;  // padding slot
    uint2 ab = d.p_ab[p];
    if (is_dyn(ab.y)) continue;
    const uint32_t sid = d.sid[ab.x];
    const SceneGeo &G = k.geo[sid];
    if ((ab.y & ~TDS_STATIC) < 1u + G.nwall) continue;
    float4 rn = d.p_rn[p], L0 = d.p_la[p];
    float2 L1 = d.p_lb[p];
    float3 n = f3(rn), t1, t2;
    onb(n, t1, t2);
    float3 F = (1.0f / k.dt) * (L0.x * n + L0.y * t1 + L0.z * t2);
    float3 xc = f3(d.pos[ab.x]) + rn.w * n;
    float3 arm = xc - make_float3(G.tp[0], G.tp[1], G.tp[2]);
    float3 T = cross(arm, F) + (1.0f / k.dt) * make_float3(L0.w, L1.x, L1.y);
    if (k.nscenes > 1) {  // batches: per-scene accumulators
      double *dst = d.tool_acc + 6 * (size_t)sid;
      atomicAdd(dst + 0, (double)F.x); atomicAdd(dst + 1, (double)F.y); atomicAdd(dst + 2, (double)F.z);
      atomicAdd(dst + 3, (double)T.x); atomicAdd(dst + 4, (double)T.y); atomicAdd(dst + 5, (double)T.z);
      continue;
    }
    acc[0] += F.x; acc[1] += F.y; acc[2] += F.z;
    acc[3] += T.x; acc[4] += T.y; acc[5] += T.z;
  }
  for (int q = 0; q < 6; ++q) {
    double t = block_sum(acc[q], sh);
    if (threadIdx.x == 0) d.dpart[6 * blockIdx.x + q] = t;
  }
}

__global__ void k_tool_final(DevPtrs d, uint32_t nscenes) {
  if (step_failed(d)) return;
  if (nscenes == 1) {
    if (threadIdx.x < 6) {
      double t = 0.0;
      for (int b = 0; b < kToolBlocks; ++b) t += d.dpart[6 * b + threadIdx.x];
      d.tool_out[threadIdx.x] = (float)t;
    }
    return;
  }
  for (uint32_t q = threadIdx.x; q < 6 * nscenes; q += blockDim.x) {
    d.tool_out[q] = (float)d.tool_acc[q];
    d.tool_acc[q] = 0.0;
  }
}

// slot order -> particle-id order staging: x y z vx vy vz wx wy wz
__global__ void k_stage(DevPtrs d, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t id = d.pid[i];
    float4 p = d.pos[i], v = d.pv[2 * i], w = d.pv[2 * i + 1];
    d.stage[0 * (size_t)n + id] = p.x; d.stage[1 * (size_t)n + id] = p.y;
    d.stage[2 * (size_t)n + id] = p.z; d.stage[3 * (size_t)n + id] = v.x;
    d.stage[4 * (size_t)n + id] = v.y; d.stage[5 * (size_t)n + id] = v.z;
    d.stage[6 * (size_t)n + id] = w.x; d.stage[7 * (size_t)n + id] = w.y;
    d.stage[8 * (size_t)n + id] = w.z; d.stage[9 * (size_t)n + id] = p.w;
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

// The compiled solver kernels, by shape index.
using PgsKernel = void (*)(DevPtrs, SolveArgs);
template <int I>
constexpr PgsKernel pgs_kernel() {
  return k_pgs<kShapes[I][0], kShapes[I][1], kShapes[I][2]>;
}
const PgsKernel kPgsKernels[kNumShapes] = {pgs_kernel<0>(), pgs_kernel<1>(), pgs_kernel<2>(), pgs_kernel<3>(),
                                           pgs_kernel<4>(), pgs_kernel<5>()};
int g_pgs_occupancy[kNumShapes];  // co-resident CTAs per SM of each shape (tds_pgs_setup)

int tds_pgs_shapes() { return kNumShapes; }
void tds_pgs_shape(int i, int *threads, int *per_thread) {
  *threads = kShapes[i][0];
  *per_thread = kShapes[i][1];
}

cudaError_t tds_launch_pgs(const DevPtrs &d, const StepConsts &k, uint32_t max_iters, float tol,
                           uint32_t every, int apply_warm, int blocks, int sync, int shape, cudaStream_t st) {
  SolveArgs a{max_iters, every, tol, k.sig_t, k.sig_r, apply_warm, sync, k.n};
  cudaMemsetAsync(d.bar, 0, 2 * sizeof(uint32_t), st);
  if (sync) cudaMemsetAsync(d.prog, 0, sizeof(uint32_t) * kProgStride * (size_t)blocks, st);
  DevPtrs dd = d;
  void *args[] = {&dd, &a};
  const int T = kShapes[shape][0];
  return cudaLaunchCooperativeKernel((const void *)kPgsKernels[shape], dim3(blocks), dim3(T), args,
                                     pgs_smem(pgs_wave(T, kShapes[shape][1])), st);
}

cudaError_t tds_launch_impact(const DevPtrs &d, const StepConsts &k, float e, float vimp, uint32_t iters,
                              int blocks, cudaStream_t st) {
  ImpactArgs a{e, vimp, k.dt, {k.g[0], k.g[1], k.g[2]}, k.ups, k.sig_t, k.sig_r, iters};
  cudaMemsetAsync(d.bar, 0, 2 * sizeof(uint32_t), st);
  cudaMemsetAsync(d.ctr + CTR_IMPACTS, 0, sizeof(uint32_t), st);
  DevPtrs dd = d;
  void *args[] = {&dd, &a};
  return cudaLaunchCooperativeKernel((const void *)k_impact, dim3(blocks), dim3(512), args, 0, st);
}

// Opt the solver into its shared-memory stages; returns the co-resident
// blocks per SM for the cooperative launch.
int tds_pgs_setup() {
  int occ_min = 0;
  for (int i = 0; i < kNumShapes; ++i) {
    const int T = kShapes[i][0];
    const size_t smem = pgs_smem(pgs_wave(T, kShapes[i][1]));
    if (cudaFuncSetAttribute((const void *)kPgsKernels[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)kPgsKernels[i], T, smem) != cudaSuccess)
      return 0;
    g_pgs_occupancy[i] = occ;
    occ_min = i == 0 ? occ : (occ < occ_min ? occ : occ_min);
  }
  return occ_min;
}

// Co-resident CTAs per SM of compiled shape i (after tds_pgs_setup).
int tds_pgs_occupancy(int i) { return g_pgs_occupancy[i]; }

int tds_launch_finish(const DevPtrs &d, const StepConsts &k, uint32_t cap, cudaStream_t st) {
  k_writeback<<<grid_for(cap, 256), 256, 0, st>>>(d);
  k_prev_ranges<<<grid_for(k.n, 256), 256, 0, st>>>(d, k.n, cap);
  k_tool_partial<<<kToolBlocks, 256, 0, st>>>(d, k);
  k_tool_final<<<1, 256, 0, st>>>(d, k.nscenes);
  k_integrate<<<grid_for(k.n, 256), 256, 0, st>>>(d, k);
  return 5;
}

void tds_launch_stage(const DevPtrs &d, uint32_t n, cudaStream_t st) {
  k_stage<<<grid_for(n, 256), 256, 0, st>>>(d, n);
}

