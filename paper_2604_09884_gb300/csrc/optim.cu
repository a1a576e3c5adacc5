// Network description, Adam update (Sec. 4 trains with Adam) and small FP64 helpers.
#include <math.h>

#include "mlp.cuh"

namespace inrct {

int make_net(const inrct_mlp* mlp, const inrct_grid* grid, Net* n) {
  INRCT_REQUIRE(mlp, "mlp descriptor must not be NULL");
  INRCT_REQUIRE(mlp->kind == INRCT_FFN_RELU || mlp->kind == INRCT_SIREN || mlp->kind == INRCT_HASH,
                "unknown INR kind %d", mlp->kind);
  INRCT_REQUIRE(mlp->d == 2 || mlp->d == 3, "input dimension d=%d must be 2 or 3", mlp->d);
  INRCT_REQUIRE(!grid || grid->d == mlp->d, "mlp d=%d differs from grid d=%d", mlp->d,
                grid ? grid->d : 0);
  INRCT_REQUIRE(!grid || grid->fov == 0 || grid->fov == 1, "grid fov=%d must be 0 or 1", grid ? grid->fov : 0);
  n->fov = grid ? grid->fov : 0;
  INRCT_REQUIRE(mlp->n_hidden >= 1 && mlp->n_hidden + 1 <= kMaxLayers,
                "n_hidden=%d out of range (1..%d)", mlp->n_hidden, kMaxLayers - 1);
  INRCT_REQUIRE(mlp->width == 64 || mlp->width == 128 || mlp->width == 256,
                "width=%d unsupported (64, 128 or 256)", mlp->width);
  INRCT_REQUIRE(mlp->prec == INRCT_FP32 || mlp->prec == INRCT_BF16, "unknown precision %d",
                mlp->prec);
  if (mlp->kind == INRCT_FFN_RELU) {
    INRCT_REQUIRE(mlp->n_feat >= 1 && mlp->n_feat <= 2048, "n_feat=%d out of range (1..2048)",
                  mlp->n_feat);
    INRCT_REQUIRE(mlp->B != nullptr, "FFN needs the Fourier matrix B");
  } else if (mlp->kind == INRCT_SIREN) {
    INRCT_REQUIRE(mlp->omega0 > 0.f, "SIREN needs omega0 > 0");
  } else {
    INRCT_REQUIRE(mlp->hash_levels >= 1 && mlp->hash_levels <= kMaxHashLevels,
                  "hash_levels=%d out of range (1..%d)", mlp->hash_levels, kMaxHashLevels);
    const int hf = mlp->hash_feats;
    INRCT_REQUIRE(hf == 1 || hf == 2 || hf == 4 || hf == 8, "hash_feats=%d must be 1, 2, 4 or 8", hf);
    INRCT_REQUIRE(mlp->hash_levels * hf <= kMaxHashInputs, "hash_levels x hash_feats = %d exceeds %d",
                  mlp->hash_levels * hf, kMaxHashInputs);
    INRCT_REQUIRE(mlp->hash_log2_T >= 4 && mlp->hash_log2_T <= 24, "hash_log2_T=%d out of range (4..24)",
                  mlp->hash_log2_T);
    INRCT_REQUIRE(mlp->hash_base >= 1 && mlp->hash_base <= 65536, "hash_base=%d out of range (1..65536)",
                  mlp->hash_base);
    INRCT_REQUIRE(mlp->hash_growth >= 1.0 && mlp->hash_growth <= 4.0,
                  "hash_growth=%g out of range [1, 4]", mlp->hash_growth);
    INRCT_REQUIRE(mlp->prec == INRCT_FP32, "the hash-encoded INR runs on the FP32 path only");
  }
  n->hL = n->hF = n->hlog2T = 0;
  n->n_table = 0;
  if (mlp->kind == INRCT_HASH) {
    n->hL = mlp->hash_levels;
    n->hF = mlp->hash_feats;
    n->hlog2T = mlp->hash_log2_T;
    for (int l = 0; l < n->hL; ++l) {
      // N_l = floor(base * growth^l), in double precision as the definition reads
      const double r = std::floor((double)mlp->hash_base * std::pow(mlp->hash_growth, (double)l));
      INRCT_REQUIRE(r >= 1.0 && r <= (double)(1 << 20), "hash level %d resolution %g out of range (1..2^20)",
                    l, r);
      n->hres[l] = (int)r;
    }
    n->n_table = (int64_t)n->hL * ((int64_t)1 << n->hlog2T) * n->hF;
  }
  n->kind = mlp->kind;
  n->d = mlp->d;
  n->F = mlp->kind == INRCT_FFN_RELU ? mlp->n_feat : 0;
  n->W = mlp->width;
  n->L = mlp->n_hidden;
  n->omega0 = mlp->omega0;
  n->B = mlp->B;
  n->B_host = mlp->kind == INRCT_FFN_RELU ? mlp->B_host : nullptr;
  n->K0 = mlp->kind == INRCT_FFN_RELU ? 2 * mlp->n_feat
          : mlp->kind == INRCT_HASH    ? n->hL * n->hF
                                       : mlp->d;
  int64_t off = n->n_table;
  for (int l = 0; l <= n->L; ++l) {
    n->in_dim[l] = l == 0 ? n->K0 : n->W;
    n->out_dim[l] = l == n->L ? 1 : n->W;
    n->offW[l] = off;
    off += (int64_t)n->in_dim[l] * n->out_dim[l];
    n->offb[l] = off;
    off += n->out_dim[l];
  }
  n->p = off;
  return INRCT_OK;
}

// Bias-corrected step size and epsilon of Adam step t, with both corrections folded:
// lr_t = lr * sqrt(1 - b2^t) / (1 - b1^t) and eps_t = eps * sqrt(1 - b2^t), so that
// theta -= lr_t * m / (sqrt(s) + eps_t) equals lr * m_hat / (sqrt(s_hat) + eps).
// Every operation is rounded on its own (no contraction into fused multiply-adds) and
// the powers are formed by square-and-multiply, so host and device produce the same
// bits: the graph-driven batched step reads t from device memory and must agree with
// the host-driven single-problem step.
namespace {
__host__ __device__ inline double rn_mul(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  volatile double r = a * b;
  return r;
#endif
}
__host__ __device__ inline double rn_sub(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(a, -b);
#else
  volatile double r = a - b;
  return r;
#endif
}
__host__ __device__ inline double rn_sqrt(double a) {
#ifdef __CUDA_ARCH__
  return __dsqrt_rn(a);
#else
  return sqrt(a);
#endif
}
__host__ __device__ inline double rn_div(double a, double b) {
#ifdef __CUDA_ARCH__
  return __ddiv_rn(a, b);
#else
  volatile double r = a / b;
  return r;
#endif
}
__host__ __device__ inline double rn_pow(double b, long long t) {
  double r = 1.0;
  while (t > 0) {
    if (t & 1) r = rn_mul(r, b);
    b = rn_mul(b, b);
    t >>= 1;
  }
  return r;
}
__host__ __device__ inline void adam_folded(double lr, double b1, double b2, double eps, long long t,
                                            float* lr_t, float* eps_t) {
  const double bc1 = rn_sub(1.0, rn_pow(b1, t));
  const double rb2 = rn_sqrt(rn_sub(1.0, rn_pow(b2, t)));
  *lr_t = (float)rn_div(rn_mul(lr, rb2), bc1);
  *eps_t = (float)rn_mul(eps, rb2);
}

// One Adam element on values in registers (every kernel below uses this arithmetic, so
// all of them give the same bits).
__device__ __forceinline__ void adam_math(float& th, double g, float& m, float& s, float b1, float b2,
                                          float lr_t, float eps_t) {
  const float gi = (float)g;
  m = fmaf(b1, m, (1.f - b1) * gi);
  s = fmaf(b2, s, (1.f - b2) * gi * gi);
  th -= lr_t * m / (sqrtf(s) + eps_t);
}

__device__ __forceinline__ void adam_elem(float* theta, const double* g, float* m, float* s, int64_t i,
                                          float b1, float b2, float lr_t, float eps_t) {
  float th = theta[i], mi = m[i], si = s[i];
  adam_math(th, g[i], mi, si, b1, b2, lr_t, eps_t);
  m[i] = mi;
  s[i] = si;
  theta[i] = th;
}

// Four consecutive elements 4j .. 4j+3 with 16-byte accesses (the caller checked alignment).
__device__ __forceinline__ void adam_elem4(float* theta, const double* g, float* m, float* s, int64_t j,
                                           float b1, float b2, float lr_t, float eps_t) {
  float4 th = reinterpret_cast<float4*>(theta)[j];
  float4 mv = reinterpret_cast<float4*>(m)[j];
  float4 sv = reinterpret_cast<float4*>(s)[j];
  const double2 g01 = reinterpret_cast<const double2*>(g)[2 * j];
  const double2 g23 = reinterpret_cast<const double2*>(g)[2 * j + 1];
  adam_math(th.x, g01.x, mv.x, sv.x, b1, b2, lr_t, eps_t);
  adam_math(th.y, g01.y, mv.y, sv.y, b1, b2, lr_t, eps_t);
  adam_math(th.z, g23.x, mv.z, sv.z, b1, b2, lr_t, eps_t);
  adam_math(th.w, g23.y, mv.w, sv.w, b1, b2, lr_t, eps_t);
  reinterpret_cast<float4*>(m)[j] = mv;
  reinterpret_cast<float4*>(s)[j] = sv;
  reinterpret_cast<float4*>(theta)[j] = th;
}

// Element range of thread i: vector path (elements 4i .. 4i+3) when vec, then the scalar tail.
__device__ __forceinline__ void adam_thread(float* theta, const double* g, float* m, float* s, int64_t p,
                                            bool vec, float b1, float b2, float lr_t, float eps_t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!vec) {
    if (i < p) adam_elem(theta, g, m, s, i, b1, b2, lr_t, eps_t);
    return;
  }
  const int64_t nv = p / 4;
  if (i < nv) adam_elem4(theta, g, m, s, i, b1, b2, lr_t, eps_t);
  else if (i - nv < p % 4) adam_elem(theta, g, m, s, 4 * nv + (i - nv), b1, b2, lr_t, eps_t);
}

bool adam_vec_ok(const float* theta, const double* g, const float* m, const float* s) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(theta) | reinterpret_cast<uintptr_t>(g) |
                      reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(s);
  return (a & 15) == 0;
}

int64_t adam_threads(int64_t p, bool vec) { return vec ? p / 4 + p % 4 : p; }
}  // namespace

__global__ void adam_kernel(float* __restrict__ theta, const double* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ s, int64_t p, int vec, float b1,
                            float b2, float lr_t, float eps_t) {
  adam_thread(theta, g, m, s, p, vec != 0, b1, b2, lr_t, eps_t);
}

// Adam with the step index read from device memory (*t, already advanced for this step).
__global__ void adam_devt_kernel(float* __restrict__ theta, const double* __restrict__ g,
                                 float* __restrict__ m, float* __restrict__ s, int64_t p, int vec, double lr,
                                 double b1, double b2, double eps, const long long* __restrict__ t) {
  __shared__ float fold[2];
  if (threadIdx.x == 0) adam_folded(lr, b1, b2, eps, *t, &fold[0], &fold[1]);
  __syncthreads();
  adam_thread(theta, g, m, s, p, vec != 0, (float)b1, (float)b2, fold[0], fold[1]);
}

__global__ void step_counter_kernel(long long* t) { *t += 1; }

__global__ void fov_zero_kernel(float* __restrict__ image, int64_t n, int N) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !in_fov(i, N)) image[i] = 0.f;
}

// Index-set check: counts[0] out of range, counts[1] outside the field of view, counts[2]
// repeats (an index whose bit in the bitmap was already set by another entry).
__global__ void check_index_kernel(const int32_t* __restrict__ idx, int64_t n_idx, int64_t n, int N, int fov,
                                   unsigned int* __restrict__ bits, unsigned long long* __restrict__ counts) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_idx) return;
  const int64_t i = idx[k];
  if (i < 0 || i >= n) {
    atomicAdd(&counts[0], 1ull);
    return;
  }
  if (fov && !in_fov(i, N)) atomicAdd(&counts[1], 1ull);
  const unsigned int b = 1u << (i & 31);
  if (atomicOr(&bits[i >> 5], b) & b) atomicAdd(&counts[2], 1ull);
}

size_t check_index_ws_bytes(int64_t n) { return 256 + align_up(sizeof(unsigned int) * ((n + 31) / 32), 256); }

int check_index_set(const int32_t* idx, int64_t n_idx, int64_t n, int N, int fov, void* ws, size_t ws_bytes,
                    long long* counts_out, cudaStream_t st) {
  const size_t need = check_index_ws_bytes(n);
  if (!ws || ws_bytes < need) {
    set_error("inrct_check_index_set: workspace of %zu bytes too small (need %zu)", ws_bytes, need);
    return INRCT_ERR_WORKSPACE;
  }
  unsigned long long* counts = static_cast<unsigned long long*>(ws);
  unsigned int* bits = reinterpret_cast<unsigned int*>(static_cast<char*>(ws) + 256);
  cudaError_t e = cudaMemsetAsync(ws, 0, need, st);
  if (e == cudaSuccess && n_idx > 0) {
    check_index_kernel<<<ceil_div(n_idx, 256), 256, 0, st>>>(idx, n_idx, n, N, fov, bits, counts);
    e = cudaGetLastError();
  }
  unsigned long long h[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error("inrct_check_index_set: %s", cudaGetErrorString(e));
    return INRCT_ERR_CUDA;
  }
  for (int q = 0; q < 3; ++q) counts_out[q] = (long long)h[q];
  return INRCT_OK;
}

int fov_zero(float* image, int64_t n, int N, cudaStream_t st) {
  fov_zero_kernel<<<ceil_div(n, 256), 256, 0, st>>>(image, n, N);
  INRCT_CHECK_LAUNCH("field-of-view mask");
  return INRCT_OK;
}

int adam_update(float* theta, const double* grad, float* m, float* s, int64_t p,
                const inrct_adam* a, cudaStream_t st) {
  INRCT_REQUIRE(a->t >= 1, "Adam step index t must be >= 1");
  INRCT_REQUIRE(m && s, "Adam moments must not be NULL");
  float lr_t, eps_t;
  adam_folded(a->lr, a->beta1, a->beta2, a->eps, a->t, &lr_t, &eps_t);
  const bool vec = adam_vec_ok(theta, grad, m, s);
  adam_kernel<<<ceil_div(adam_threads(p, vec), 256), 256, 0, st>>>(theta, grad, m, s, p, vec, (float)a->beta1,
                                                                   (float)a->beta2, lr_t, eps_t);
  INRCT_CHECK_LAUNCH("adam");
  return INRCT_OK;
}

int adam_update_devt(float* theta, const double* grad, float* m, float* s, int64_t p,
                     const inrct_adam* a, const long long* t_dev, cudaStream_t st) {
  INRCT_REQUIRE(m && s && t_dev, "Adam moments and the step counter must not be NULL");
  const bool vec = adam_vec_ok(theta, grad, m, s);
  adam_devt_kernel<<<ceil_div(adam_threads(p, vec), 256), 256, 0, st>>>(theta, grad, m, s, p, vec, a->lr,
                                                                        a->beta1, a->beta2, a->eps, t_dev);
  INRCT_CHECK_LAUNCH("adam (device step index)");
  return INRCT_OK;
}

int advance_step_counter(long long* t_dev, cudaStream_t st) {
  step_counter_kernel<<<1, 1, 0, st>>>(t_dev);
  INRCT_CHECK_LAUNCH("step counter");
  return INRCT_OK;
}

__global__ void f64_to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

int f64_to_f32(const double* in, float* out, int64_t n, cudaStream_t st) {
  f64_to_f32_kernel<<<ceil_div(n, 256), 256, 0, st>>>(in, out, n);
  INRCT_CHECK_LAUNCH("f64 to f32");
  return INRCT_OK;
}

}  // namespace inrct
