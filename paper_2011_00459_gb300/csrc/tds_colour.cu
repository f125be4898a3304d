// tds_colour.cu -- greedy colouring of the contact graph and the stable
// re-ordering of the contact rows into colour order.
//
// Two contacts are adjacent when they share a dynamic particle (static
// surfaces never couple contacts). Every contact gets the smallest colour not
// used by an adjacent contact of higher priority, priority being the
// SplitMix64 hash of its key. This is exactly sequential greedy colouring in
// decreasing priority order; on the GPU it is computed Jones-Plassmann style
// by a persistent kernel that walks the priority DAG in rounds: a contact is
// coloured as soon as all its higher-priority neighbours are, then releases
// its lower-priority neighbours. Contacts of one colour touch disjoint
// particles, so a colour is one parallel Gauss-Seidel step.
#include "tds_internal.cuh"

namespace {

__device__ __forceinline__ bool is_dyn(uint32_t b) { return (b & TDS_STATIC) == 0u; }

__global__ void k_inc_count(DevPtrs d) {
  const uint32_t nc = d.ctr[CTR_NC];
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    uint2 ab = d.c_ab[c];
    atomicAdd(d.inc_cnt + ab.x, 1u);
    if (is_dyn(ab.y)) atomicAdd(d.inc_cnt + ab.y, 1u);
  }
}

__global__ void k_inc_fill(DevPtrs d) {
  const uint32_t nc = d.ctr[CTR_NC];
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    uint2 ab = d.c_ab[c];
    d.inc_list[atomicAdd(d.inc_cursor + ab.x, 1u)] = c;
    if (is_dyn(ab.y)) d.inc_list[atomicAdd(d.inc_cursor + ab.y, 1u)] = c;
  }
}

// wait[c] = number of neighbours of higher priority; sources start round 0.
__global__ void k_colour_init(DevPtrs d) {
  const uint32_t nc = d.ctr[CTR_NC];
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    uint2 ab = d.c_ab[c];
    unsigned long long pc = priority(d.c_key[c]);
    int32_t w = 0;
    uint32_t ends[2] = {ab.x, ab.y};
    for (int e = 0; e < 2; ++e) {
      if (!is_dyn(ends[e])) continue;
      for (uint32_t m = d.inc_start[ends[e]]; m < d.inc_start[ends[e] + 1]; ++m) {
        uint32_t o = d.inc_list[m];
        if (o != c && priority(d.c_key[o]) > pc) ++w;
      }
    }
    d.wait[c] = w;
    d.colour[c] = TDS_NO_COLOUR;
    if (w == 0) {
      uint32_t q = atomicAdd(d.ctr + CTR_FCOUNT, 1u);
      if (q < nc) d.frontier0[q] = c;
    }
  }
}

// Persistent, co-resident launch: one round per grid barrier.
__global__ void k_colour_rounds(DevPtrs d) {
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t nc = d.ctr[CTR_NC];
  __shared__ uint32_t s_maxcol;
  if (threadIdx.x == 0) s_maxcol = 0;
  __syncthreads();
  for (uint32_t round = 0;; ++round) {
    uint32_t *cur = (round & 1) ? d.frontier1 : d.frontier0;
    uint32_t *nxt = (round & 1) ? d.frontier0 : d.frontier1;
    volatile uint32_t *fc = d.ctr + CTR_FCOUNT;
    const uint32_t ncur = min(fc[round % 3], nc);
    uint32_t *push = d.ctr + CTR_FCOUNT + (round + 1) % 3;
    if (blockIdx.x == 0 && threadIdx.x == 0) d.ctr[CTR_FCOUNT + (round + 2) % 3] = 0u;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < ncur; idx += stride) {
      uint32_t c = __ldcg(cur + idx);
      uint2 ab = d.c_ab[c];
      unsigned long long pc = priority(d.c_key[c]);
      unsigned long long used0 = 0ull, used1 = 0ull;
      uint32_t ends[2] = {ab.x, ab.y};
      for (int e = 0; e < 2; ++e) {
        if (!is_dyn(ends[e])) continue;
        for (uint32_t m = d.inc_start[ends[e]]; m < d.inc_start[ends[e] + 1]; ++m) {
          uint32_t o = d.inc_list[m];
          if (o == c || priority(d.c_key[o]) < pc) continue;
          uint32_t col = __ldcg(d.colour + o);
          if (col < 64) used0 |= 1ull << col;
          else if (col < 128) used1 |= 1ull << (col - 64);
        }
      }
      uint32_t col;
      if (~used0) col = __ffsll((long long)~used0) - 1;
      else if (~used1) col = 64 + __ffsll((long long)~used1) - 1;
      else { col = TDS_MAX_COLOURS - 1; latch_error(d.err, DEV_ERR_CAPACITY); }
      __stcg(d.colour + c, (uint8_t)col);
      atomicMax(&s_maxcol, col + 1);
      __threadfence();
      for (int e = 0; e < 2; ++e) {
        if (!is_dyn(ends[e])) continue;
        for (uint32_t m = d.inc_start[ends[e]]; m < d.inc_start[ends[e] + 1]; ++m) {
          uint32_t o = d.inc_list[m];
          if (o == c || priority(d.c_key[o]) > pc) continue;
          if (atomicSub(d.wait + o, 1) == 1) {
            uint32_t q = atomicAdd(push, 1u);
            if (q < nc) nxt[q] = o;
          }
        }
      }
    }
    if (!grid_barrier(d.bar, d.err)) return;
    if (fc[(round + 1) % 3] == 0u || round > nc) break;
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(d.ctr + CTR_NCOL, s_maxcol);
}

// ---- stable counting sort of contacts by bucket = 2 colour + static? ------
// Colours are < TDS_MAX_COLOURS once the colouring finished; a contact left
// uncoloured (only after a latched error) is clamped into the last bucket.
__device__ __forceinline__ uint32_t bucket_of(const DevPtrs &d, uint32_t c) {
  uint32_t col = d.colour[c];
  if (col >= TDS_MAX_COLOURS) col = TDS_MAX_COLOURS - 1;
  return 2u * col + (is_dyn(d.c_ab[c].y) ? 0u : 1u);
}

__global__ void k_bucket_hist(DevPtrs d) {
  __shared__ uint32_t hist[TDS_NBUCKETS];
  const uint32_t nc = d.ctr[CTR_NC];
  for (uint32_t b = threadIdx.x; b < TDS_NBUCKETS; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  uint32_t base = blockIdx.x * TDS_TILE;
  for (uint32_t k = threadIdx.x; k < TDS_TILE; k += blockDim.x) {
    uint32_t c = base + k;
    if (c < nc) {
      if (d.colour[c] >= TDS_MAX_COLOURS) latch_error(d.err, DEV_ERR_CAPACITY);
      atomicAdd(hist + bucket_of(d, c), 1u);
    }
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < TDS_NBUCKETS; b += blockDim.x)
    d.tile_hist[b * d.ntiles + blockIdx.x] = hist[b];
}

__global__ void k_bucket_starts(DevPtrs d) {
  for (uint32_t b = threadIdx.x; b <= TDS_NBUCKETS; b += blockDim.x)
    d.bucket_start[b] = b < TDS_NBUCKETS ? d.tile_off[b * d.ntiles] : d.ctr[CTR_NC];
}

// Scatter every contact's rows to its colour-order position: tile offset of
// its bucket + rank among equal buckets earlier in the tile (warp match +
// per-warp counts), so the order inside a bucket is the owner order.
__global__ void __launch_bounds__(256) k_bucket_scatter(DevPtrs d) {
  constexpr int W = 8;  // warps per block
  __shared__ uint32_t base[TDS_NBUCKETS];
  __shared__ uint32_t wcnt[W][TDS_NBUCKETS];
  const uint32_t nc = d.ctr[CTR_NC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t b = threadIdx.x; b < TDS_NBUCKETS; b += blockDim.x)
    base[b] = d.tile_off[b * d.ntiles + blockIdx.x];
  for (uint32_t chunk = 0; chunk < TDS_TILE; chunk += 256) {
    for (uint32_t q = threadIdx.x; q < W * TDS_NBUCKETS; q += blockDim.x) (&wcnt[0][0])[q] = 0;
    __syncthreads();
    uint32_t c = blockIdx.x * TDS_TILE + chunk + threadIdx.x;
    bool live = c < nc;
    uint32_t bk = live ? bucket_of(d, c) : 0xFFFFFFFFu;
    uint32_t peers = __match_any_sync(0xffffffffu, bk);
    uint32_t rank_in_warp = __popc(peers & ((1u << lane) - 1u));
    if (live && rank_in_warp == 0) wcnt[warp][bk] = __popc(peers);
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < TDS_NBUCKETS; b += blockDim.x) {
      uint32_t run = base[b];
      for (int w = 0; w < W; ++w) { uint32_t t = wcnt[w][b]; wcnt[w][b] = run; run += t; }
      base[b] = run;
    }
    __syncthreads();
    if (live) {
      uint32_t p = wcnt[warp][bk] + rank_in_warp;
      d.order[p] = c;
      d.p_ab[p] = d.c_ab[c];
      d.p_rn[p] = d.c_rn[c];
      d.p_rq[p] = d.c_rq[c];
      d.p_rm[p] = d.c_rm[c];
      if (bk & 1u) { d.p_sv[p] = d.c_sv[c]; d.p_sw[p] = d.c_sw[c]; }
      d.p_la[p] = d.c_la[c];
      d.p_lb[p] = d.c_lb[c];
    }
    __syncthreads();
  }
}

}  // namespace

int tds_launch_colouring(const DevPtrs &d, uint32_t n, uint32_t cap, int coop_blocks,
                         int coop_threads, cudaStream_t st) {
  unsigned gc = (cap + 255) / 256;
  if (gc > 152 * 16) gc = 152 * 16;
  if (gc == 0) gc = 1;
  cudaMemsetAsync(d.inc_cnt, 0, sizeof(uint32_t) * (n + 1), st);
  k_inc_count<<<gc, 256, 0, st>>>(d);
  tds_scan_exclusive(d.inc_cnt, d.inc_start, n, d.scan_tmp, st);
  cudaMemcpyAsync(d.inc_cursor, d.inc_start, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
  k_inc_fill<<<gc, 256, 0, st>>>(d);
  cudaMemsetAsync(d.ctr + CTR_FCOUNT, 0, 3 * sizeof(uint32_t), st);
  cudaMemsetAsync(d.ctr + CTR_NCOL, 0, sizeof(uint32_t), st);
  k_colour_init<<<gc, 256, 0, st>>>(d);
  cudaMemsetAsync(d.bar, 0, 2 * sizeof(uint32_t), st);
  DevPtrs dd = d;
  void *args[] = {&dd};
  cudaLaunchCooperativeKernel((const void *)k_colour_rounds, dim3(coop_blocks), dim3(coop_threads),
                              args, 0, st);
  k_bucket_hist<<<d.ntiles, 256, 0, st>>>(d);
  tds_scan_exclusive(d.tile_hist, d.tile_off, TDS_NBUCKETS * d.ntiles, d.scan_tmp, st);
  k_bucket_starts<<<1, 256, 0, st>>>(d);
  k_bucket_scatter<<<d.ntiles, 256, 0, st>>>(d);
  return 12;
}

const void *tds_colour_kernel() { return (const void *)k_colour_rounds; }
