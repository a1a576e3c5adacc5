// Ramp filter F of the filtered least-squares loss (Sec. 2):
//   L_FLS(z, y) = 1/2 (z - y)^T F (z - y),  dL/dz = F (z - y)   (Sec. 3, after Algorithm 1).
// F convolves every detector row (fixed view, and fixed detector row v for the
// cone) along the bin axis with the band-limited ramp (Ram-Lak) kernel of the
// textbook FBP, sampled at the bin pitch tau = du * (2/N) at the isocentre:
//   (F r)_b = tau * sum_k h[k] r_{b-k},  h[0] = 1/(4 tau^2),
//   h[k] = -1/(pi^2 k^2 tau^2) for odd k, 0 for even k != 0;
// bins outside the detector count as zero.  F is symmetric, so the same
// kernel gives the gradient.  One block per detector row; the row and the
// kernel taps are staged in shared memory.
#include <math.h>

#include "filter.cuh"
#include "projector.cuh"

namespace inrct {

__global__ void ramp_kernel(const float* __restrict__ r, float* __restrict__ out, int A, float tau,
                            double* __restrict__ loss_part) {
  extern __shared__ float sh[];
  float* row = sh;      // [A]
  float* h = sh + A;    // [A]: h[k] for k = 0..A-1
  const int64_t base = (int64_t)blockIdx.x * A;
  const float inv_t2 = 1.f / (tau * tau);
  for (int b = threadIdx.x; b < A; b += blockDim.x) {
    row[b] = r[base + b];
    h[b] = b == 0 ? 0.25f * inv_t2 : ((b & 1) ? -inv_t2 / (float)(M_PI * M_PI * (double)b * b) : 0.f);
  }
  __syncthreads();
  float lsum = 0.f;
  for (int b = threadIdx.x; b < A; b += blockDim.x) {
    float acc = h[0] * row[b];
    for (int k = 1; k < A; k += 2) {
      const float left = b - k >= 0 ? row[b - k] : 0.f;
      const float right = b + k < A ? row[b + k] : 0.f;
      acc = fmaf(h[k], left + right, acc);
    }
    acc *= tau;
    out[base + b] = acc;
    lsum = fmaf(row[b], acc, lsum);
  }
  __shared__ float red[32];
  for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    loss_part[blockIdx.x] = 0.5 * s;
  }
}

__global__ void reduce_partials_kernel(const double* __restrict__ in, int64_t n, double* __restrict__ out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += in[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

static int64_t ramp_rows(const inrct_geom* g) {
  return (int64_t)g->n_views * (g->kind == INRCT_CONE3D ? g->n_bins_v : 1);
}

size_t ramp_ws_bytes(const inrct_geom* geom) {
  return align_up(sizeof(double) * ramp_rows(geom), 256) + 256;
}

int ramp_filter_impl(const inrct_geom* geom, const inrct_grid* grid, const float* r, float* out,
                     double* loss_out, void* ws, size_t ws_bytes, cudaStream_t st) {
  INRCT_TRY(check_geom(geom, grid));
  INRCT_REQUIRE(r && out && loss_out, "r, out and loss_out must not be NULL");
  INRCT_REQUIRE(r != out, "ramp filter cannot run in place");
  INRCT_REQUIRE(geom->n_bins_u <= 6144, "ramp filter supports at most 6144 bins per row");
  const size_t need = ramp_ws_bytes(geom);
  if (!ws || ws_bytes < need) {
    set_error("ramp filter: workspace of %zu bytes too small (need %zu)", ws_bytes, need);
    return INRCT_ERR_WORKSPACE;
  }
  const int64_t rows = ramp_rows(geom);
  const int A = geom->n_bins_u;
  const float tau = (float)(geom->du * 2.0 / grid->N);
  double* part = static_cast<double*>(ws);
  ramp_kernel<<<(unsigned)rows, 256, sizeof(float) * 2 * A, st>>>(r, out, A, tau, part);
  INRCT_CHECK_LAUNCH("ramp filter");
  reduce_partials_kernel<<<1, 1024, 0, st>>>(part, rows, loss_out);
  INRCT_CHECK_LAUNCH("ramp loss reduce");
  return INRCT_OK;
}

}  // namespace inrct
