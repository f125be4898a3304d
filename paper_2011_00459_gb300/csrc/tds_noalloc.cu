// tds_noalloc.cu -- tds_find_pair_contacts_noalloc: the particle-pair contact
// search of tds_step (sorted-cell broadphase + the bit-exact FP32 pair
// predicate) as a standalone call that allocates no memory.
//
// Some callers cannot let a library allocate device memory: a simulator
// stepping inside a fixed-rate real-time loop, where cudaMalloc/cudaFree may
// synchronize the device and stall the frame, or a host application whose
// device memory is entirely owned by its own pool allocator with a fixed
// budget. This call takes the caller's input and output buffers and keeps all
// of its intermediate arrays in one file-scope __device__ array of fixed size
// (below), which every GPU that loads the library holds until the process
// exits.
//
// Properties of the shared scratch array:
//  * Host code cannot use the array's name as a device address; the first call
//    on each device looks the address up with cudaGetSymbolAddress (with that
//    device current) and caches it. That first call should therefore come
//    before any stream capture.
//  * Every call reuses the same array and leaves its contents behind; what must
//    start at zero (the cell counters) is cleared by each call on its stream.
//  * Calls whose GPU work overlaps (on different streams, or from different
//    host threads) race on the array; serialize them on one stream.
//  * The cached address belongs to the device's primary context: after the
//    caller resets the device (cudaDeviceReset), it is stale.
//  * The order of the output keys depends only on the input: every cell's
//    particles are sorted by index, whatever its size.
#include <mutex>
#include <string>

#include "tds_internal.cuh"

namespace {

constexpr uint32_t kMaxN = TDS_NOALLOC_MAX_PARTICLES;
constexpr uint32_t kMaxCells = 262144u;

constexpr size_t align64(size_t w) { return (w + 63) & ~(size_t)63; }  // 256-byte regions
constexpr size_t kPlan = 0;
constexpr size_t kCellCount = kPlan + 64;
constexpr size_t kCellStart = kCellCount + align64(kMaxCells + 1);
constexpr size_t kCursor = kCellStart + align64(kMaxCells + 1);
constexpr size_t kCellOf = kCursor + align64(kMaxCells);
constexpr size_t kPerm = kCellOf + align64(kMaxN);
constexpr size_t kSPos = kPerm + align64(kMaxN);
constexpr size_t kSId = kSPos + align64(4 * (size_t)kMaxN);
constexpr size_t kCnt = kSId + align64(kMaxN);
constexpr size_t kCStart = kCnt + align64(kMaxN + 1);
constexpr size_t kTmp = kCStart + align64(kMaxN + 1);
constexpr size_t kTotalWords = kTmp + align64(kMaxCells / 2048 + 64);

// The scratch array (about 5.3 MB).
static __device__ __align__(256) uint32_t g_noalloc_scratch[kTotalWords];

struct Plan {
  float lo[3];
  float inv;
  int gnx, gny, gnz;
  int cohesive;
};

struct View {
  uint32_t *base;
  __device__ Plan *plan() const { return reinterpret_cast<Plan *>(base + kPlan); }
  __device__ uint32_t *cell_count() const { return base + kCellCount; }
  __device__ uint32_t *cell_start() const { return base + kCellStart; }
  __device__ uint32_t *cursor() const { return base + kCursor; }
  __device__ uint32_t *cell_of() const { return base + kCellOf; }
  __device__ uint32_t *perm() const { return base + kPerm; }
  __device__ float4 *spos() const { return reinterpret_cast<float4 *>(base + kSPos); }
  __device__ uint32_t *sid() const { return base + kSId; }
  __device__ uint32_t *cnt() const { return base + kCnt; }
  __device__ uint32_t *cstart() const { return base + kCStart; }
};

// Same FP32 pair predicate as the step (explicit round-to-nearest, this
// association, strict comparison).
__device__ __forceinline__ bool touch(float4 A, float4 B, int cohesive) {
  float dx = __fsub_rn(B.x, A.x), dy = __fsub_rn(B.y, A.y), dz = __fsub_rn(B.z, A.z);
  float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  float rs = __fadd_rn(A.w, B.w);
  float R = cohesive ? __fadd_rn(rs, __fmul_rn(0.025f, rs)) : rs;
  return d2 < __fmul_rn(R, R);
}

__device__ __forceinline__ int axis_cell(float x, float x0, float inv, int n) {
  float t = floorf((x - x0) * inv);
  if (!(t >= 0.0f)) return 0;
  if (t >= (float)(n - 1)) return n - 1;
  return (int)t;
}

// One block: bounding box, largest radius, and a grid of at most kMaxCells
// cells, each wider than any contact reach.
__global__ void k_plan(View v, const float *x, const float *y, const float *z, const float *r,
                       uint32_t n, int cohesive) {
  __shared__ float sh[7][32];
  float m[7] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.f};
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    float p[3] = {x[i], y[i], z[i]};
    for (int a = 0; a < 3; ++a) { m[a] = fminf(m[a], p[a]); m[3 + a] = fmaxf(m[3 + a], p[a]); }
    m[6] = fmaxf(m[6], r[i]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < 7; ++q) {
    float t = m[q];
    for (int o = 16; o > 0; o >>= 1) {
      float u = __shfl_down_sync(0xffffffffu, t, o);
      t = (q < 3) ? fminf(t, u) : fmaxf(t, u);
    }
    if (lane == 0) sh[q][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int q = 0; q < 7; ++q) {
      float t = sh[q][0];
      for (int w = 1; w < nw; ++w) t = (q < 3) ? fminf(t, sh[q][w]) : fmaxf(t, sh[q][w]);
      m[q] = t;
    }
    float cell = 2.0f * m[6] * 1.025f * 1.02f;
    if (!(cell > 0.f)) cell = 1.f;
    int dims[3];
    for (;;) {
      unsigned long long tot = 1;
      for (int a = 0; a < 3; ++a) {
        dims[a] = (int)ceilf((m[3 + a] - m[a]) / cell) + 1;
        tot *= (unsigned long long)dims[a];
      }
      if (tot <= kMaxCells) break;
      cell *= 1.25f;
    }
    Plan *P = v.plan();
    for (int a = 0; a < 3; ++a) P->lo[a] = m[a];
    P->inv = 1.0f / cell;
    P->gnx = dims[0]; P->gny = dims[1]; P->gnz = dims[2];
    P->cohesive = cohesive;
  }
}

__global__ void k_cells(View v, const float *x, const float *y, const float *z, uint32_t n) {
  const Plan P = *v.plan();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int cx = axis_cell(x[i], P.lo[0], P.inv, P.gnx);
    int cy = axis_cell(y[i], P.lo[1], P.inv, P.gny);
    int cz = axis_cell(z[i], P.lo[2], P.inv, P.gnz);
    uint32_t c = ((uint32_t)cz * P.gny + cy) * P.gnx + cx;
    v.cell_of()[i] = c;
    atomicAdd(v.cell_count() + c, 1u);
  }
}

__global__ void k_scatter(View v, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v.perm()[atomicAdd(v.cursor() + v.cell_of()[i], 1u)] = i;
}

// Reproducible order inside each cell, whatever the order of the atomic
// scatter: ascending particle index. Cells of up to kSmallCell particles are
// sorted by one thread each (insertion sort), larger ones by k_cell_sort_big.
constexpr uint32_t kSmallCell = 64;

__global__ void k_cell_sort(View v) {
  const Plan P = *v.plan();
  const uint32_t ncells = (uint32_t)P.gnx * P.gny * P.gnz;
  uint32_t *perm = v.perm();
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    uint32_t s = v.cell_start()[c], e = v.cell_start()[c + 1];
    if (e - s < 2 || e - s > kSmallCell) continue;
    for (uint32_t a = s + 1; a < e; ++a) {
      uint32_t val = perm[a], b = a;
      while (b > s && perm[b - 1] > val) { perm[b] = perm[b - 1]; --b; }
      perm[b] = val;
    }
  }
}

// Cells with more than kSmallCell particles (a grid that k_plan coarsened
// because of a far outlier puts thousands of particles in one cell): one
// block per cell sorts its m entries in place with a bitonic network in the
// form whose every comparator puts the smaller value at the lower index
// (each merge stage starts by comparing mirrored positions of its blocks,
// then halves). Comparators that reach past m are skipped, which is the same
// as padding the sequence to a power of two with values larger than any
// index. Every block walks the cells in a fixed stride; all threads of a
// block read the same bounds, so the block decides together.
__global__ void __launch_bounds__(1024) k_cell_sort_big(View v) {
  const Plan P = *v.plan();
  const uint32_t ncells = (uint32_t)P.gnx * P.gny * P.gnz;
  uint32_t *perm = v.perm();
  for (uint32_t c = blockIdx.x; c < ncells; c += gridDim.x) {
    const uint32_t s = v.cell_start()[c], e = v.cell_start()[c + 1];
    const uint32_t m = e - s;
    if (m <= kSmallCell) continue;
    uint32_t *a = perm + s;
    uint32_t pow2 = 1;
    while (pow2 < m) pow2 <<= 1;
    const uint32_t half = pow2 >> 1;
    for (uint32_t k = 2; k <= pow2; k <<= 1) {
      const uint32_t hk = k >> 1;
      for (uint32_t t = threadIdx.x; t < half; t += blockDim.x) {  // mirrored pairs of each k-block
        const uint32_t blk = t / hk, x = t % hk;
        const uint32_t i = blk * k + x, j = blk * k + (k - 1u - x);
        if (j < m) {
          const uint32_t ai = a[i], aj = a[j];
          if (ai > aj) { a[i] = aj; a[j] = ai; }
        }
      }
      __syncthreads();
      for (uint32_t d = k >> 2; d > 0; d >>= 1) {  // half-cleaners at distance d
        for (uint32_t t = threadIdx.x; t < half; t += blockDim.x) {
          const uint32_t i = (t / d) * 2u * d + (t % d), j = i + d;
          if (j < m) {
            const uint32_t ai = a[i], aj = a[j];
            if (ai > aj) { a[i] = aj; a[j] = ai; }
          }
        }
        __syncthreads();
      }
    }
  }
}

__global__ void k_gather(View v, const float *x, const float *y, const float *z, const float *r,
                         uint32_t n) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    uint32_t i = v.perm()[j];
    v.spos()[j] = make_float4(x[i], y[i], z[i], r[i]);
    v.sid()[j] = i;
  }
}

template <bool kWrite>
__global__ void k_pairs(View v, uint32_t n, unsigned long long *keys, uint32_t cap) {
  const Plan P = *v.plan();
  const float4 *sp = v.spos();
  const uint32_t *sid = v.sid();
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const float4 A = sp[j];
    const uint32_t me = sid[j];
    int cx = axis_cell(A.x, P.lo[0], P.inv, P.gnx);
    int cy = axis_cell(A.y, P.lo[1], P.inv, P.gny);
    int cz = axis_cell(A.z, P.lo[2], P.inv, P.gnz);
    int x0 = max(cx - 1, 0), x1 = min(cx + 1, P.gnx - 1);
    uint32_t found = 0, out = kWrite ? v.cstart()[j] : 0u;
    for (int zz = max(cz - 1, 0); zz <= min(cz + 1, P.gnz - 1); ++zz)
      for (int yy = max(cy - 1, 0); yy <= min(cy + 1, P.gny - 1); ++yy) {
        uint32_t row = ((uint32_t)zz * P.gny + yy) * P.gnx;
        uint32_t s = v.cell_start()[row + x0], e = v.cell_start()[row + x1 + 1];
        for (uint32_t k = s; k < e; ++k) {
          uint32_t other = sid[k];
          if (other <= me || !touch(A, sp[k], P.cohesive)) continue;
          if (kWrite) {
            if (out < cap) keys[out] = ((unsigned long long)me << 32) | other;
            ++out;
          } else {
            ++found;
          }
        }
      }
    if (!kWrite) v.cnt()[j] = found;
  }
}

__global__ void k_total(View v, uint32_t n, uint32_t *count_out) { *count_out = v.cstart()[n]; }

std::mutex g_mu;
uint32_t *g_base[256];  // device address of the scratch array, per device ordinal

}  // namespace

tds_status tds_set_error_message(tds_status s, const char *msg);  // tds_api.cu

extern "C" tds_status tds_find_pair_contacts_noalloc(const float *x, const float *y, const float *z,
                                                     const float *radius, uint32_t n, int32_t cohesive,
                                                     uint64_t *keys, uint32_t cap, uint32_t *count,
                                                     void *stream) {
  if (!x || !y || !z || !radius || !keys || !count)
    return tds_set_error_message(TDS_ERR_INVALID_ARG, "tds_find_pair_contacts_noalloc: NULL pointer");
  if (n == 0)
    return tds_set_error_message(TDS_ERR_INVALID_ARG, "tds_find_pair_contacts_noalloc: n must be >= 1");
  if (n > kMaxN)
    return tds_set_error_message(TDS_ERR_CAPACITY,
                                 "tds_find_pair_contacts_noalloc: n exceeds TDS_NOALLOC_MAX_PARTICLES (65536)");
  // an error left pending by an earlier call of the caller is reported, and
  // left pending, rather than blamed on this call's launches
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess)
    return tds_set_error_message(TDS_ERR_CUDA, (std::string("tds_find_pair_contacts_noalloc: a CUDA error of an "
                                                            "earlier call is pending: ") +
                                                    cudaGetErrorString(e)).c_str());
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256)
    return tds_set_error_message(TDS_ERR_CUDA, "tds_find_pair_contacts_noalloc: cudaGetDevice failed");
  uint32_t *base;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return tds_set_error_message(TDS_ERR_CUDA,
                                     "tds_find_pair_contacts_noalloc: cudaGetSymbolAddress failed");
      g_base[dev] = static_cast<uint32_t *>(p);
    }
    base = g_base[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  View v{base};
  const unsigned grid = (n + 255) / 256;
  e = cudaMemsetAsync(base + kCellCount, 0, sizeof(uint32_t) * (kMaxCells + 1), st);
  if (e != cudaSuccess)
    return tds_set_error_message(TDS_ERR_CUDA, (std::string("tds_find_pair_contacts_noalloc: cudaMemsetAsync: ") +
                                                    cudaGetErrorString(e)).c_str());
  k_plan<<<1, 1024, 0, st>>>(v, x, y, z, radius, n, cohesive ? 1 : 0);
  k_cells<<<grid, 256, 0, st>>>(v, x, y, z, n);
  tds_scan_exclusive(base + kCellCount, base + kCellStart, kMaxCells, base + kTmp, st);
  e = cudaMemcpyAsync(base + kCursor, base + kCellStart, sizeof(uint32_t) * kMaxCells,
                      cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess)
    return tds_set_error_message(TDS_ERR_CUDA, (std::string("tds_find_pair_contacts_noalloc: cudaMemcpyAsync: ") +
                                                    cudaGetErrorString(e)).c_str());
  k_scatter<<<grid, 256, 0, st>>>(v, n);
  k_cell_sort<<<kMaxCells / 256, 256, 0, st>>>(v);
  k_cell_sort_big<<<128, 1024, 0, st>>>(v);
  k_gather<<<grid, 256, 0, st>>>(v, x, y, z, radius, n);
  k_pairs<false><<<(n + 127) / 128, 128, 0, st>>>(v, n, nullptr, 0);
  tds_scan_exclusive(base + kCnt, base + kCStart, n, base + kTmp, st);
  k_pairs<true><<<(n + 127) / 128, 128, 0, st>>>(v, n, reinterpret_cast<unsigned long long *>(keys), cap);
  k_total<<<1, 1, 0, st>>>(v, n, count);
  // the launches above are the only work since the pending-error check on
  // entry, so an error now is theirs
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return tds_set_error_message(TDS_ERR_CUDA, (std::string("tds_find_pair_contacts_noalloc: launch: ") +
                                                    cudaGetErrorString(e)).c_str());
  return TDS_OK;
}
