// tds_aggregate.cu -- aggregate bodies of active zones (section "Macroscale
// model", Eqs. aggregate_mass to aggregate_rot_vel): per zone the mass,
// centre of mass, velocity, inertia tensor about the centre of mass and the
// angular velocity I^+ L of the particles it contains. Two passes, as in the
// definition: (1) membership, M, sum m x, sum m v; (2) the second moments and
// angular momentum about the centre of mass. FP64 accumulation; each thread
// walks a contiguous run of slots (spatially sorted, so zones change rarely)
// and flushes its running sums into shared memory when the zone changes.
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

template <int K>
__device__ __forceinline__ void flush(double *sh, int z, const double *acc) {
  if (z < 0) return;
#pragma unroll
  for (int j = 0; j < K; ++j)
    if (acc[j] != 0.0) atomicAdd(sh + z * K + j, acc[j]);
}

template <int K>
__device__ __forceinline__ void block_to_global(double *sh, double *sums, uint32_t nz) {
  __syncthreads();
  for (uint32_t q = threadIdx.x; q < nz * K; q += blockDim.x)
    if (sh[q] != 0.0) atomicAdd(sums + q, sh[q]);
}

__global__ void __launch_bounds__(kAggThreads) k_agg_first(DevPtrs d, uint32_t n, const tds_zone *zones,
                                                           uint32_t nz, uint8_t *zone_id, double *sums) {
  __shared__ tds_zone sz[TDS_MAX_ZONES];
  __shared__ double sh[TDS_MAX_ZONES * kFirst];
  for (uint32_t q = threadIdx.x; q < nz * sizeof(tds_zone) / 4; q += blockDim.x)
    reinterpret_cast<uint32_t *>(sz)[q] = reinterpret_cast<const uint32_t *>(zones)[q];
  for (uint32_t q = threadIdx.x; q < nz * kFirst; q += blockDim.x) sh[q] = 0.0;
  __syncthreads();
  const uint32_t nt = gridDim.x * blockDim.x, t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t per = (n + nt - 1) / nt;
  const uint32_t i0 = min(n, t * per), i1 = min(n, i0 + per);
  double acc[kFirst] = {};
  int cur = -1;
  for (uint32_t i = i0; i < i1; ++i) {
    const float4 p = d.pos[i];
    const int z = zone_of(sz, nz, d.sid[i], p);
    zone_id[i] = z < 0 ? 0xFF : (uint8_t)z;
    if (z < 0) continue;
    if (z != cur) {
      flush<kFirst>(sh, cur, acc);
#pragma unroll
      for (int j = 0; j < kFirst; ++j) acc[j] = 0.0;
      cur = z;
    }
    const float4 v = d.pv[2 * (size_t)i];
    const double m = 1.0 / (double)v.w;
    acc[0] += m;
    acc[1] += m * p.x; acc[2] += m * p.y; acc[3] += m * p.z;
    acc[4] += m * v.x; acc[5] += m * v.y; acc[6] += m * v.z;
    acc[7] += 1.0;
  }
  flush<kFirst>(sh, cur, acc);
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
  const uint32_t nt = gridDim.x * blockDim.x, t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t per = (n + nt - 1) / nt;
  const uint32_t i0 = min(n, t * per), i1 = min(n, i0 + per);
  double acc[kSecond] = {};
  int cur = -1;
  for (uint32_t i = i0; i < i1; ++i) {
    const uint8_t zb = zone_id[i];
    if (zb == 0xFF) continue;
    const int z = zb;
    if (z != cur) {
      flush<kSecond>(sh, cur, acc);
#pragma unroll
      for (int j = 0; j < kSecond; ++j) acc[j] = 0.0;
      cur = z;
    }
    const float4 p = d.pos[i];
    const float4 v = d.pv[2 * (size_t)i];
    const double m = 1.0 / (double)v.w;
    const double dx = (double)p.x - com[z][0], dy = (double)p.y - com[z][1], dz = (double)p.z - com[z][2];
    acc[0] += m * dx * dx; acc[1] += m * dy * dy; acc[2] += m * dz * dz;
    acc[3] += m * dx * dy; acc[4] += m * dx * dz; acc[5] += m * dy * dz;
    acc[6] += m * (dy * v.z - dz * v.y);
    acc[7] += m * (dz * v.x - dx * v.z);
    acc[8] += m * (dx * v.y - dy * v.x);
  }
  flush<kSecond>(sh, cur, acc);
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
  uint32_t blocks = (n + 8u * kAggThreads - 1) / (8u * kAggThreads);  // ~8 slots per thread
  if (blocks < 1) blocks = 1;
  if (blocks > (uint32_t)(8 * sms)) blocks = 8 * sms;
  k_agg_first<<<blocks, kAggThreads, 0, st>>>(d, n, zones, nz, zone_id, first);
  k_agg_second<<<blocks, kAggThreads, 0, st>>>(d, n, nz, zone_id, first, second);
  k_agg_final<<<1, TDS_MAX_ZONES, 0, st>>>(nz, first, second, out);
  return 3;
}

size_t tds_aggregate_sums_words() { return (size_t)TDS_MAX_ZONES * (kFirst + kSecond); }
