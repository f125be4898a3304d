// tds_aggregate.cu -- aggregate bodies of active zones (section "Macroscale
// model", Eqs. aggregate_mass to aggregate_rot_vel): per zone the mass,
// centre of mass, velocity, inertia tensor about the centre of mass and the
// angular velocity I^+ L of the particles it contains. Two passes, as in the
// definition: (1) membership, M, sum m x, sum m v; (2) the second moments and
// angular momentum about the centre of mass. FP64 accumulation, reduced warp
// by warp (see WarpSums).
#include "tds_internal.cuh"

namespace {

constexpr int kAggThreads = 256;
constexpr int kFirst = 8;   // m, m x (3), m v (3), count
constexpr int kSecond = 9;  // m dx dx^T (6: xx yy zz xy xz yz), m dx x v (3)

// First zone of the particle's scene containing p (-1: none); the FP32
// half-space test in the documented operation order.
__device__ __forceinline__ int zone_of(const tds_zone *zones, uint32_t nz, uint32_t sid, float4 p) {
  for (uint32_t z = 0; z < nz; ++z) {
    const tds_zone &Z = zones[z];
    if (Z.scene != sid) continue;
    bool in = true;
    for (uint32_t k = 0; k < Z.n_planes && in; ++k) {
      const float *q = Z.planes[k];
      const float s = __fadd_rn(__fadd_rn(__fmul_rn(q[0], p.x), __fmul_rn(q[1], p.y)), __fmul_rn(q[2], p.z));
      in = s <= q[3];
    }
    if (in) return (int)z;
  }
  return -1;
}

// Warp-synchronous accumulation of K sums per zone. Each warp walks its own
// contiguous stretch of slots, 32 consecutive particles per iteration
// (coalesced). When every particle of the iteration that lies in a zone lies
// in the same zone (the usual case: slot order is spatial) the warp reduces
// the K values with shuffles and lane c keeps component c of the running sum
// of the warp's current zone, flushed into shared memory when the zone
// changes; iterations that straddle zones add lane by lane.
template <int K>
struct WarpSums {
  int cur = -1;
  double acc = 0.0;  // lane c < K: component c for zone cur
  __device__ void flush(double *sh, int lane) {
    if (cur >= 0 && lane < K && acc != 0.0) atomicAdd(sh + cur * K + lane, acc);
    acc = 0.0;
  }
  __device__ void add(double *sh, int lane, int z, const double (&val)[K]) {
    const unsigned full = 0xffffffffu;
    const int zsel = __reduce_max_sync(full, z);
    if (zsel < 0) return;
    const bool uniform = __all_sync(full, z < 0 || z == zsel);
    if (!uniform) {
      if (z >= 0)
#pragma unroll
        for (int c = 0; c < K; ++c)
          if (val[c] != 0.0) atomicAdd(sh + z * K + c, val[c]);
      return;
    }
    if (zsel != cur) {
      flush(sh, lane);
      cur = zsel;
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
      double t = val[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(full, t, o);
      if (lane == c) acc += t;
    }
  }
};

template <int K>
__device__ __forceinline__ void block_to_global(double *sh, double *sums, uint32_t nz) {
  __syncthreads();
  for (uint32_t q = threadIdx.x; q < nz * K; q += blockDim.x)
    if (sh[q] != 0.0) atomicAdd(sums + q, sh[q]);
}

// The stretch [lo, hi) of slots of this warp (a multiple of 32 long).
__device__ __forceinline__ void warp_stretch(uint32_t n, uint32_t &lo, uint32_t &hi) {
  const uint32_t nw = gridDim.x * (blockDim.x >> 5), w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint32_t per = (n + nw - 1) / nw;
  per = (per + 31u) & ~31u;
  lo = min(n, w * per);
  hi = min(n, lo + per);
}

__global__ void __launch_bounds__(kAggThreads) k_agg_first(DevPtrs d, uint32_t n, const tds_zone *zones,
                                                           uint32_t nz, uint8_t *zone_id, double *sums) {
  __shared__ tds_zone sz[TDS_MAX_ZONES];
  __shared__ double sh[TDS_MAX_ZONES * kFirst];
  for (uint32_t q = threadIdx.x; q < nz * sizeof(tds_zone) / 4; q += blockDim.x)
    reinterpret_cast<uint32_t *>(sz)[q] = reinterpret_cast<const uint32_t *>(zones)[q];
  for (uint32_t q = threadIdx.x; q < nz * kFirst; q += blockDim.x) sh[q] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  uint32_t lo, hi;
  warp_stretch(n, lo, hi);
  WarpSums<kFirst> ws;
  for (uint32_t base = lo; base < hi; base += 32) {
    const uint32_t i = base + lane;
    int z = -1;
    double val[kFirst] = {};
    if (i < hi) {
      const float4 p = d.pos[i];
      z = p.w > 0.0f ? zone_of(sz, nz, d.sid[i], p) : -1;  // dormant slots belong to no zone
      zone_id[i] = z < 0 ? 0xFF : (uint8_t)z;
      if (z >= 0) {
        const float4 v = d.pv[2 * (size_t)i];
        const double m = 1.0 / (double)v.w;
        val[0] = m;
        val[1] = m * p.x; val[2] = m * p.y; val[3] = m * p.z;
        val[4] = m * v.x; val[5] = m * v.y; val[6] = m * v.z;
        val[7] = 1.0;
      }
    }
    ws.add(sh, lane, z, val);
  }
  ws.flush(sh, lane);
  block_to_global<kFirst>(sh, sums, nz);
}

__global__ void __launch_bounds__(kAggThreads) k_agg_second(DevPtrs d, uint32_t n, uint32_t nz,
                                                            const uint8_t *zone_id, const double *first,
                                                            double *sums) {
  __shared__ double com[TDS_MAX_ZONES][3];
  __shared__ double sh[TDS_MAX_ZONES * kSecond];
  for (uint32_t z = threadIdx.x; z < nz; z += blockDim.x) {
    const double M = first[z * kFirst];
    for (int a = 0; a < 3; ++a) com[z][a] = M > 0.0 ? first[z * kFirst + 1 + a] / M : 0.0;
  }
  for (uint32_t q = threadIdx.x; q < nz * kSecond; q += blockDim.x) sh[q] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  uint32_t lo, hi;
  warp_stretch(n, lo, hi);
  WarpSums<kSecond> ws;
  for (uint32_t base = lo; base < hi; base += 32) {
    const uint32_t i = base + lane;
    int z = -1;
    double val[kSecond] = {};
    if (i < hi && zone_id[i] != 0xFF) {
      z = zone_id[i];
      const float4 p = d.pos[i];
      const float4 v = d.pv[2 * (size_t)i];
      const double m = 1.0 / (double)v.w;
      const double dx = (double)p.x - com[z][0], dy = (double)p.y - com[z][1], dz = (double)p.z - com[z][2];
      val[0] = m * dx * dx; val[1] = m * dy * dy; val[2] = m * dz * dz;
      val[3] = m * dx * dy; val[4] = m * dx * dz; val[5] = m * dy * dz;
      val[6] = m * (dy * v.z - dz * v.y);
      val[7] = m * (dz * v.x - dx * v.z);
      val[8] = m * (dx * v.y - dy * v.x);
    }
    ws.add(sh, lane, z, val);
  }
  ws.flush(sh, lane);
  block_to_global<kSecond>(sh, sums, nz);
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations
// (Jacobi's method: zero one off-diagonal entry at a time); A becomes
// diagonal, V holds the eigenvectors as columns.
__device__ void jacobi3(double A[3][3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
    const double scale = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]);
    if (off <= 1e-300 || off <= 1e-17 * scale) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
        for (int k = 0; k < 3; ++k) {  // A <- A J
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // A <- J^T A
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {  // V <- V J
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

__global__ void k_agg_final(uint32_t nz, const double *first, const double *second, tds_aggregate *out) {
  const uint32_t z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nz) return;
  tds_aggregate o{};
  const double *F = first + z * kFirst, *S = second + z * kSecond;
  const double M = F[0];
  if (M > 0.0) {
    o.count = (uint32_t)F[7];
    o.mass = M;
    for (int a = 0; a < 3; ++a) {
      o.com[a] = F[1 + a] / M;
      o.vel[a] = F[4 + a] / M;
    }
    // I = tr(S) 1 - S with S the second moment about the centre of mass
    const double tr = S[0] + S[1] + S[2];
    double I[3][3] = {{tr - S[0], -S[3], -S[4]}, {-S[3], tr - S[1], -S[5]}, {-S[4], -S[5], tr - S[2]}};
    o.inertia[0] = I[0][0]; o.inertia[1] = I[1][1]; o.inertia[2] = I[2][2];
    o.inertia[3] = I[0][1]; o.inertia[4] = I[0][2]; o.inertia[5] = I[1][2];
    // the momentum about the centre of mass of the velocities relative to v_A
    // equals sum m dx x v, since sum m dx = 0
    const double L[3] = {S[6], S[7], S[8]};
    double V[3][3];
    jacobi3(I, V);
    const double lam[3] = {I[0][0], I[1][1], I[2][2]};
    const double lmax = fmax(fabs(lam[0]), fmax(fabs(lam[1]), fabs(lam[2])));
    for (int k = 0; k < 3; ++k) {
      if (!(fabs(lam[k]) > 1e-12 * lmax)) continue;  // pseudo-inverse: skip null directions
      const double proj = (V[0][k] * L[0] + V[1][k] * L[1] + V[2][k] * L[2]) / lam[k];
      for (int a = 0; a < 3; ++a) o.omega[a] += proj * V[a][k];
    }
  }
  out[z] = o;
}

}  // namespace

int tds_launch_aggregate(const DevPtrs &d, uint32_t n, const tds_zone *zones, uint32_t nz, uint8_t *zone_id,
                         double *sums, tds_aggregate *out, cudaStream_t st) {
  double *first = sums, *second = sums + (size_t)TDS_MAX_ZONES * kFirst;
  cudaMemsetAsync(sums, 0, sizeof(double) * TDS_MAX_ZONES * (kFirst + kSecond), st);
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // 8 blocks per SM (the warps walk stretches of ~n / (64 SMs) slots), fewer
  // for small n so that every warp has at least 128 slots
  uint32_t blocks = (n + 128u * (kAggThreads / 32) - 1) / (128u * (kAggThreads / 32));
  if (blocks < 1) blocks = 1;
  if (blocks > (uint32_t)(8 * sms)) blocks = 8 * sms;
  k_agg_first<<<blocks, kAggThreads, 0, st>>>(d, n, zones, nz, zone_id, first);
  k_agg_second<<<blocks, kAggThreads, 0, st>>>(d, n, nz, zone_id, first, second);
  k_agg_final<<<1, TDS_MAX_ZONES, 0, st>>>(nz, first, second, out);
  return 3;
}

size_t tds_aggregate_sums_words() { return (size_t)TDS_MAX_ZONES * (kFirst + kSecond); }
