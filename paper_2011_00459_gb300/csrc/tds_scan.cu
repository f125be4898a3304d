// tds_scan.cu -- exclusive prefix sums of uint32 counts (cell occupancy,
// contacts per particle, incidences per particle, bucket histograms), built
// from warp-shuffle scans in three phases: tile sums, a scan of the tile
// sums, and a per-tile scan with the tile offset added.
#include "tds_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // 2048 elements per block

__device__ __forceinline__ uint32_t warp_inclusive(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the
// block total through *total.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t *total) {
  __shared__ uint32_t warp_sums[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = warp_inclusive(v);
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < kThreads / 32 ? warp_sums[lane] : 0u;
    uint32_t si = warp_inclusive(s);
    if (lane < kThreads / 32) warp_sums[lane] = si - s;
    if (lane == kThreads / 32 - 1) warp_sums[kThreads / 32] = si;  // total
  }
  __syncthreads();
  uint32_t excl = inc - v + warp_sums[warp];
  *total = warp_sums[kThreads / 32];
  __syncthreads();
  return excl;
}

__global__ void k_tile_sums(const uint32_t *__restrict__ in, uint32_t m, uint32_t *__restrict__ sums) {
  size_t base = (size_t)blockIdx.x * kTile + threadIdx.x * kItems;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    size_t i = base + k;
    if (i < m) s += in[i];
  }
  uint32_t total;
  (void)block_exclusive(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block scans the tile sums in chunks (tile counts are small).
__global__ void k_scan_sums(uint32_t *sums, uint32_t ntiles) {
  uint32_t carry = 0;
  for (uint32_t base = 0; base < ntiles; base += kThreads) {
    uint32_t i = base + threadIdx.x;
    uint32_t v = i < ntiles ? sums[i] : 0u;
    uint32_t total;
    uint32_t e = block_exclusive(v, &total);
    if (i < ntiles) sums[i] = e + carry;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[ntiles] = carry;
}

__global__ void k_tile_scan(const uint32_t *in, uint32_t m, const uint32_t *sums,
                            uint32_t ntiles, uint32_t *out) {
  size_t base = (size_t)blockIdx.x * kTile + threadIdx.x * kItems;
  uint32_t v[kItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    size_t i = base + k;
    v[k] = i < m ? in[i] : 0u;
    s += v[k];
  }
  uint32_t total;
  uint32_t run = block_exclusive(s, &total) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    size_t i = base + k;
    if (i < m) out[i] = run;
    run += v[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[m] = sums[ntiles];
}

}  // namespace

size_t tds_scan_tmp_words(uint32_t m) { return (size_t)(m + kTile - 1) / kTile + 2; }

// out[0..m] = exclusive prefix sums of in[0..m), out[m] = total. In-place
// (in == out) is allowed. tmp holds tds_scan_tmp_words(m) words.
void tds_scan_exclusive(const uint32_t *in, uint32_t *out, uint32_t m, uint32_t *tmp,
                        cudaStream_t st) {
  uint32_t ntiles = (m + kTile - 1) / kTile;
  if (ntiles == 0) {
    cudaMemsetAsync(out, 0, sizeof(uint32_t), st);
    return;
  }
  k_tile_sums<<<ntiles, kThreads, 0, st>>>(in, m, tmp);
  k_scan_sums<<<1, kThreads, 0, st>>>(tmp, ntiles);
  k_tile_scan<<<ntiles, kThreads, 0, st>>>(in, m, tmp, ntiles, out);
}
