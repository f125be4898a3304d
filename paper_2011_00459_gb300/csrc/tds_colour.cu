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

// Incidence counts per particle (the priorities were written with the
// contacts).
__global__ void k_inc_count(DevPtrs d) {
  const uint32_t nc = d.ctr[CTR_NC];
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    uint2 ab = d.c_ab[c];
    atomicAdd(d.inc_cnt + ab.x, 1u);
    if (is_dyn(ab.y)) atomicAdd(d.inc_cnt + ab.y, 1u);
  }
}

// Incidence entries carry the contact id and the high word of its priority,
// so walking a neighbourhood needs no dependent loads to compare priorities.
__global__ void k_inc_fill(DevPtrs d) {
  const uint32_t nc = d.ctr[CTR_NC];
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    uint2 ab = d.c_ab[c];
    uint32_t hi = (uint32_t)(d.prio[c] >> 32);
    d.inc_ent[atomicAdd(d.inc_cursor + ab.x, 1u)] = make_uint2(c, hi);
    if (is_dyn(ab.y)) d.inc_ent[atomicAdd(d.inc_cursor + ab.y, 1u)] = make_uint2(c, hi);
  }
}

// Is neighbour entry e of higher priority than contact c (priority pc)?
// The high words decide unless they tie; then the full priorities do.
__device__ __forceinline__ bool higher(const DevPtrs &d, uint2 e, unsigned long long pc) {
  uint32_t hc = (uint32_t)(pc >> 32);
  if (e.y != hc) return e.y > hc;
  return d.prio[e.x] > pc;
}

constexpr int kBatch = 8;

// A slot in a frontier list for each calling lane: one atomic per group of
// converged lanes instead of one per lane (the frontier counter is a single
// address that every released contact would otherwise hit).
__device__ __forceinline__ uint32_t frontier_slot(uint32_t *counter) {
  const unsigned mask = __activemask();
  const unsigned lane = threadIdx.x & 31u;
  const int leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if ((int)lane == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + (uint32_t)__popc(mask & ((1u << lane) - 1u));
}

// wait[c] = number of uncoloured neighbours of higher priority; sources
// start round 0. A full colouring starts with every contact uncoloured; an
// incremental one (see incremental_colouring) with the colours the
// narrowphase kept, which also enter the colour count.
__global__ void k_colour_init(DevPtrs d) {
  const uint32_t nc = d.ctr[CTR_NC];
  const bool inc = incremental_colouring(d);
  __shared__ uint32_t s_maxcol;
  if (threadIdx.x == 0) s_maxcol = 0;
  __syncthreads();
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    if (inc) {
      const uint32_t kept = d.colour[c];
      if (kept != TDS_NO_COLOUR) {
        atomicMax(&s_maxcol, kept + 1u);
        continue;
      }
    }
    uint2 ab = d.c_ab[c];
    unsigned long long pc = d.prio[c];
    int32_t w = 0;
    uint32_t ends[2] = {ab.x, ab.y};
    for (int k = 0; k < 2; ++k) {
      if (!is_dyn(ends[k])) continue;
      const uint32_t s = d.inc_start[ends[k]], e = d.inc_start[ends[k] + 1];
      for (uint32_t m0 = s; m0 < e; m0 += kBatch) {
        uint2 ent[kBatch];
#pragma unroll
        for (int q = 0; q < kBatch; ++q) ent[q] = m0 + q < e ? d.inc_ent[m0 + q] : make_uint2(c, 0u);
#pragma unroll
        for (int q = 0; q < kBatch; ++q)
          w += (ent[q].x != c && higher(d, ent[q], pc) && (!inc || d.colour[ent[q].x] == TDS_NO_COLOUR)) ? 1 : 0;
      }
    }
    d.wait[c] = w;
    if (!inc) d.colour[c] = TDS_NO_COLOUR;
    if (w == 0) {
      const uint32_t q = frontier_slot(d.ctr + CTR_FCOUNT);
      if (q < nc) d.frontier0[q] = c;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_maxcol) atomicMax(d.ctr + CTR_NCOL, s_maxcol);
}

// Persistent, co-resident launch: one round per grid barrier. A round colours
// every contact whose higher-priority neighbours are all coloured, then
// releases its lower-priority neighbours into the next round's frontier.
__global__ void k_colour_rounds(DevPtrs d) {
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t nc = d.ctr[CTR_NC];
  const bool inc = incremental_colouring(d);
  __shared__ uint32_t s_maxcol;
  if (threadIdx.x == 0) s_maxcol = 0;
  __syncthreads();
  uint32_t round = 0, gen = 0;
  for (;; ++round) {
    uint32_t *cur = (round & 1) ? d.frontier1 : d.frontier0;
    uint32_t *nxt = (round & 1) ? d.frontier0 : d.frontier1;
    volatile uint32_t *fc = d.ctr + CTR_FCOUNT;
    const uint32_t ncur = min(fc[round % 3], nc);
    uint32_t *push = d.ctr + CTR_FCOUNT + (round + 1) % 3;
    if (blockIdx.x == 0 && threadIdx.x == 0) d.ctr[CTR_FCOUNT + (round + 2) % 3] = 0u;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < ncur; idx += stride) {
      const uint32_t c = __ldcg(cur + idx);
      const uint2 ab = d.c_ab[c];
      const unsigned long long pc = d.prio[c];
      unsigned long long used0 = 0ull, used1 = 0ull;
      const uint32_t ends[2] = {ab.x, ab.y};
      // colours of the higher-priority neighbours (all coloured already)
      for (int k = 0; k < 2; ++k) {
        if (!is_dyn(ends[k])) continue;
        const uint32_t s = d.inc_start[ends[k]], e = d.inc_start[ends[k] + 1];
        for (uint32_t m0 = s; m0 < e; m0 += kBatch) {
          uint2 ent[kBatch];
          uint32_t col[kBatch];
#pragma unroll
          for (int q = 0; q < kBatch; ++q) ent[q] = m0 + q < e ? d.inc_ent[m0 + q] : make_uint2(c, 0u);
#pragma unroll
          // a full colouring reads its higher-priority neighbours (all
          // coloured by now); an incremental one also the kept colours of
          // lower priority (its uncoloured neighbours read as no colour)
          for (int q = 0; q < kBatch; ++q)
            col[q] = (ent[q].x != c && (inc || higher(d, ent[q], pc))) ? (uint32_t)__ldcg(d.colour + ent[q].x) : 0xFFu;
#pragma unroll
          for (int q = 0; q < kBatch; ++q) {
            if (col[q] < 64) used0 |= 1ull << col[q];
            else if (col[q] < 128) used1 |= 1ull << (col[q] - 64);
          }
        }
      }
      uint32_t col;
      if (~used0) col = __ffsll((long long)~used0) - 1;
      else if (~used1) col = 64 + __ffsll((long long)~used1) - 1;
      else { col = TDS_MAX_COLOURS - 1; latch_error(d.err, DEV_ERR_CAPACITY); }
      __stcg(d.colour + c, (uint8_t)col);
      atomicMax(&s_maxcol, col + 1);
      // release the lower-priority neighbours (they read this colour in a
      // later round, after the grid barrier has published it)
      for (int k = 0; k < 2; ++k) {
        if (!is_dyn(ends[k])) continue;
        const uint32_t s = d.inc_start[ends[k]], e = d.inc_start[ends[k] + 1];
        for (uint32_t m0 = s; m0 < e; m0 += kBatch) {
          uint2 ent[kBatch];
          int32_t old[kBatch];
#pragma unroll
          for (int q = 0; q < kBatch; ++q) ent[q] = m0 + q < e ? d.inc_ent[m0 + q] : make_uint2(c, 0u);
#pragma unroll
          // (an incremental colouring releases only uncoloured neighbours:
          // a kept contact waits for nothing)
          for (int q = 0; q < kBatch; ++q)
            old[q] = (ent[q].x != c && !higher(d, ent[q], pc) &&
                      (!inc || __ldcg(d.colour + ent[q].x) == TDS_NO_COLOUR))
                         ? atomicSub(d.wait + ent[q].x, 1)
                         : 0;
#pragma unroll
          for (int q = 0; q < kBatch; ++q)
            if (old[q] == 1) {
              const uint32_t slot = frontier_slot(push);
              if (slot < nc) nxt[slot] = ent[q].x;
            }
        }
      }
    }
    if (!grid_barrier(d.bar, d.err, gen, d.wait_ns)) return;
    if (fc[(round + 1) % 3] == 0u || round > nc) break;
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(d.ctr + CTR_NCOL, s_maxcol);
  if (blockIdx.x == 0 && threadIdx.x == 0) d.ctr[CTR_ROUNDS] = round + 1;
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

// Bucket ranges in the padded colour order: every bucket starts at a multiple
// of 4 contacts (16-byte aligned rows for bulk copies); padding slots carry
// order == 0xFFFFFFFF and are never solved.
__global__ void k_bucket_starts(DevPtrs d) {
  if (threadIdx.x != 0) return;
  uint32_t run = 0;
  for (uint32_t b = 0; b < TDS_NBUCKETS; ++b) {
    uint32_t u0 = d.tile_off[b * d.ntiles];
    uint32_t u1 = b + 1 < TDS_NBUCKETS ? d.tile_off[(b + 1) * d.ntiles] : d.ctr[CTR_NC];
    uint32_t cnt = u1 - u0;
    d.bstart[b] = run;
    d.bend[b] = run + cnt;
    d.bpad[b] = run - u0;
    run += (cnt + 3u) & ~3u;
  }
  d.bstart[TDS_NBUCKETS] = run;
  d.ctr[CTR_PADDED] = run;
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
      uint32_t p = wcnt[warp][bk] + rank_in_warp + d.bpad[bk];
      d.order[p] = c;
      d.p_ab[p] = d.c_ab[c];
      d.p_rn[p] = d.c_rn[c];
      d.p_rq[p] = d.c_rq[c];
      d.p_rm[p] = d.c_rm[c];
      if (bk & 1u) { d.p_sv[p] = d.c_sv[c]; d.p_sw[p] = d.c_sw[c]; }
      d.p_la[p] = d.c_la[c];
      d.p_lb[p] = d.c_lb[c];
      if (d.nscenes > 1) atomicAdd(d.scq_cnt + (size_t)d.sid[d.c_ab[c].x] * TDS_NBUCKETS + bk, 1u);
    }
    __syncthreads();
  }
}

// Residual chunks. Inside a bucket the contacts keep the owner order, which
// is scene-major (slots are sorted by cell, cells by scene), so each scene's
// contacts of a bucket form one range; its start is the bucket's start plus
// the contacts of the earlier scenes. Each range is cut into chunks of at
// most TDS_RES_CHUNK contacts, numbered scene-major (scene, bucket, piece):
// a scene's chunks are consecutive, and they are the same chunks whether the
// scene is stepped alone or in a batch. One block.
__global__ void __launch_bounds__(1024) k_scene_chunks(DevPtrs d) {
  constexpr uint32_t NB = TDS_NBUCKETS;
  const uint32_t S = d.nscenes, total = S * NB;
  __shared__ uint32_t part[1024];
  for (uint32_t b = threadIdx.x; b < NB; b += blockDim.x) {
    uint32_t run = d.bstart[b];
    for (uint32_t q = 0; q < S; ++q) {
      const size_t e = (size_t)q * NB + b;
      const uint32_t cnt = S == 1 ? d.bend[b] - d.bstart[b] : d.scq_cnt[e];
      if (S == 1) d.scq_cnt[e] = cnt;
      d.scq_start[e] = run;
      run += cnt;
    }
  }
  __syncthreads();
  // exclusive scan of the pieces over (scene, bucket): each thread a
  // contiguous segment, then a scan of the segment sums
  const uint32_t seg = (total + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = min(threadIdx.x * seg, total), hi = min(lo + seg, total);
  uint32_t sum = 0;
  for (uint32_t e = lo; e < hi; ++e) sum += (d.scq_cnt[e] + TDS_RES_CHUNK - 1u) / TDS_RES_CHUNK;
  part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (uint32_t t = 0; t < blockDim.x; ++t) {
      const uint32_t v = part[t];
      part[t] = run;
      run += v;
    }
    d.scq_chunk[total] = run;
    d.ctr[CTR_NCHUNK] = run;
  }
  __syncthreads();
  uint32_t base = part[threadIdx.x];
  for (uint32_t e = lo; e < hi; ++e) {
    d.scq_chunk[e] = base;
    const uint32_t cnt = d.scq_cnt[e], start = d.scq_start[e], q = e / NB;
    for (uint32_t k = 0; k * TDS_RES_CHUNK < cnt; ++k)
      d.chunk[base + k] = make_uint4(start + k * TDS_RES_CHUNK, min(TDS_RES_CHUNK, cnt - k * TDS_RES_CHUNK), q, 0u);
    base += (cnt + TDS_RES_CHUNK - 1u) / TDS_RES_CHUNK;
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
  return 8;
}

// Contact rows (and initial impulses) into the padded colour order.
int tds_launch_bucketing(const DevPtrs &d, uint32_t cap, cudaStream_t st) {
  k_bucket_hist<<<d.ntiles, 256, 0, st>>>(d);
  tds_scan_exclusive(d.tile_hist, d.tile_off, TDS_NBUCKETS * d.ntiles, d.scan_tmp, st);
  k_bucket_starts<<<1, 32, 0, st>>>(d);
  cudaMemsetAsync(d.order, 0xFF, sizeof(uint32_t) * ((size_t)cap + TDS_ORDER_PAD), st);
  cudaMemsetAsync(d.p_ab, 0xFF, sizeof(uint2) * ((size_t)cap + TDS_ORDER_PAD), st);  // padding sentinel
  if (d.nscenes > 1) cudaMemsetAsync(d.scq_cnt, 0, sizeof(uint32_t) * (size_t)d.nscenes * TDS_NBUCKETS, st);
  k_bucket_scatter<<<d.ntiles, 256, 0, st>>>(d);
  k_scene_chunks<<<1, 1024, 0, st>>>(d);
  return 5;
}

const void *tds_colour_kernel() { return (const void *)k_colour_rounds; }
