// tds_fields.cu -- coarse-grained fields of the particles on a voxel grid
// (section "Coarse-graining", Eq. cg_velocity) and the conserved upwind
// advection of fluidized mass (Eq. advection).
#include <cmath>

#include "tds_internal.cuh"

tds_status tds_set_error_message(tds_status s, const char *msg);

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int voxel_axis(float x, float o, float l0, uint32_t n) {
  const float t = floorf(__fdiv_rn(__fsub_rn(x, o), l0));
  if (!(t >= 0.0f)) return 0;
  if (t >= (float)(n - 1)) return (int)n - 1;
  return (int)t;
}

// Scatter of every particle of the grid's scene into rho and p.
__global__ void k_cg_scatter(DevPtrs d, uint32_t n, tds_grid g, int kernel, float R, float *rho, float *p) {
  const float vol = g.l0 * g.l0 * g.l0;
  const float inv2R2 = kernel ? 1.0f / (2.0f * R * R) : 0.0f;
  const float norm = kernel ? 1.0f / (powf(2.5066282746310002f * R, 3.0f)) : 0.0f;  // (sqrt(2 pi) R)^-3
  const float cut2 = 9.0f * R * R;
  const int reach = kernel ? (int)ceilf(3.0f * R / g.l0) + 1 : 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (d.sid[i] != g.scene) continue;
    const float4 x = d.pos[i];
    if (x.w == 0.0f) continue;  // dormant reserve slot
    const float4 v = d.pv[2 * (size_t)i];
    const float m = 1.0f / v.w;
    const int ci = voxel_axis(x.x, g.origin[0], g.l0, g.nx);
    const int cj = voxel_axis(x.y, g.origin[1], g.l0, g.ny);
    const int ck = voxel_axis(x.z, g.origin[2], g.l0, g.nz);
    if (kernel == 0) {
      const size_t q = ((size_t)ck * g.ny + cj) * g.nx + ci;
      const float w = m / vol;
      atomicAdd(rho + q, w);
      atomicAdd(p + 3 * q, w * v.x);
      atomicAdd(p + 3 * q + 1, w * v.y);
      atomicAdd(p + 3 * q + 2, w * v.z);
      continue;
    }
    for (int k = max(ck - reach, 0); k <= min(ck + reach, (int)g.nz - 1); ++k) {
      const float dz = g.origin[2] + ((float)k + 0.5f) * g.l0 - x.z;
      for (int j = max(cj - reach, 0); j <= min(cj + reach, (int)g.ny - 1); ++j) {
        const float dy = g.origin[1] + ((float)j + 0.5f) * g.l0 - x.y;
        for (int ii = max(ci - reach, 0); ii <= min(ci + reach, (int)g.nx - 1); ++ii) {
          const float dx = g.origin[0] + ((float)ii + 0.5f) * g.l0 - x.x;
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 > cut2) continue;
          const float w = m * norm * expf(-r2 * inv2R2);
          const size_t q = ((size_t)k * g.ny + j) * g.nx + ii;
          atomicAdd(rho + q, w);
          atomicAdd(p + 3 * q, w * v.x);
          atomicAdd(p + 3 * q + 1, w * v.y);
          atomicAdd(p + 3 * q + 2, w * v.z);
        }
      }
    }
  }
}

__global__ void k_cg_velocity(size_t nvox, const float *rho, const float *p, float *u) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nvox; q += (size_t)gridDim.x * blockDim.x) {
    const float r = rho[q];
    for (int a = 0; a < 3; ++a) u[3 * q + a] = r > 0.0f ? p[3 * q + a] / r : 0.0f;
  }
}

// Upwind flux through the face between voxels a (lower) and b (upper) along
// axis ax; both neighbours evaluate it with the same operations.
__device__ __forceinline__ float face_flux(const float *u, const float *rho, size_t a, size_t b, int ax) {
  const float uf = 0.5f * (u[3 * a + ax] + u[3 * b + ax]);
  return uf > 0.0f ? uf * rho[a] : uf * rho[b];
}

__global__ void k_advect(tds_grid g, const float *u, const float *rho, const float *src, float dt, float *out) {
  const size_t nvox = (size_t)g.nx * g.ny * g.nz;
  const size_t stride[3] = {1, g.nx, (size_t)g.nx * g.ny};
  const float c = dt / g.l0;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nvox; q += (size_t)gridDim.x * blockDim.x) {
    const uint32_t idx[3] = {(uint32_t)(q % g.nx), (uint32_t)((q / g.nx) % g.ny), (uint32_t)(q / ((size_t)g.nx * g.ny))};
    const uint32_t dim[3] = {g.nx, g.ny, g.nz};
    float net = 0.0f;  // inflow minus outflow
    for (int ax = 0; ax < 3; ++ax) {
      if (idx[ax] > 0) net += face_flux(u, rho, q - stride[ax], q, ax);
      if (idx[ax] + 1 < dim[ax]) net -= face_flux(u, rho, q, q + stride[ax], ax);
    }
    out[q] = rho[q] + c * net + (src ? dt * src[q] : 0.0f);
  }
}

int grid_blocks(size_t n) {
  size_t b = (n + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (int)b;
}

}  // namespace

int tds_launch_coarse_grain(const DevPtrs &d, uint32_t n, const tds_grid &g, int kernel, float R, float *rho,
                            float *p, float *u, cudaStream_t st) {
  const size_t nvox = (size_t)g.nx * g.ny * g.nz;
  cudaMemsetAsync(rho, 0, sizeof(float) * nvox, st);
  cudaMemsetAsync(p, 0, sizeof(float) * 3 * nvox, st);
  k_cg_scatter<<<grid_blocks(n), kThreads, 0, st>>>(d, n, g, kernel, R, rho, p);
  k_cg_velocity<<<grid_blocks(nvox), kThreads, 0, st>>>(nvox, rho, p, u);
  return 2;
}

bool tds_grid_valid(const tds_grid *g) {
  if (!g || !(g->l0 > 0.0f) || !std::isfinite(g->l0) || g->nx == 0 || g->ny == 0 || g->nz == 0) return false;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(g->origin[a])) return false;
  return (double)g->nx * g->ny * g->nz < 4.0e9;
}

extern "C" tds_status tds_advect_fluid(const tds_grid *grid, const float *u, const float *rho_f,
                                       const float *source, float dt, float *rho_out, void *stream) {
  if (!tds_grid_valid(grid)) return tds_set_error_message(TDS_ERR_INVALID_ARG, "invalid grid");
  if (!u || !rho_f || !rho_out) return tds_set_error_message(TDS_ERR_INVALID_ARG, "NULL field");
  if (rho_out == rho_f) return tds_set_error_message(TDS_ERR_INVALID_ARG, "rho_out must not alias rho_f");
  if (!(dt >= 0.0f) || !std::isfinite(dt)) return tds_set_error_message(TDS_ERR_INVALID_ARG, "dt must be >= 0");
  const size_t nvox = (size_t)grid->nx * grid->ny * grid->nz;
  k_advect<<<grid_blocks(nvox), kThreads, 0, (cudaStream_t)stream>>>(*grid, u, rho_f, source, dt, rho_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return tds_set_error_message(TDS_ERR_CUDA, cudaGetErrorString(e));
  return TDS_OK;
}
