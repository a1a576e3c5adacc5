// Network description, Adam update (Sec. 4 trains with Adam) and small FP64 helpers.
#include <math.h>

#include "mlp.cuh"

namespace inrct {

int make_net(const inrct_mlp* mlp, const inrct_grid* grid, Net* n) {
  INRCT_REQUIRE(mlp, "mlp descriptor must not be NULL");
  INRCT_REQUIRE(mlp->kind == INRCT_FFN_RELU || mlp->kind == INRCT_SIREN, "unknown INR kind %d",
                mlp->kind);
  INRCT_REQUIRE(mlp->d == 2 || mlp->d == 3, "input dimension d=%d must be 2 or 3", mlp->d);
  INRCT_REQUIRE(!grid || grid->d == mlp->d, "mlp d=%d differs from grid d=%d", mlp->d,
                grid ? grid->d : 0);
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
  } else {
    INRCT_REQUIRE(mlp->omega0 > 0.f, "SIREN needs omega0 > 0");
  }
  n->kind = mlp->kind;
  n->d = mlp->d;
  n->F = mlp->kind == INRCT_FFN_RELU ? mlp->n_feat : 0;
  n->W = mlp->width;
  n->L = mlp->n_hidden;
  n->omega0 = mlp->omega0;
  n->B = mlp->B;
  n->K0 = mlp->kind == INRCT_FFN_RELU ? 2 * mlp->n_feat : mlp->d;
  int64_t off = 0;
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

__global__ void adam_kernel(float* __restrict__ theta, const double* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ s, int64_t p, float b1,
                            float b2, float lr_t, float eps_t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p) return;
  const float gi = (float)g[i];
  const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
  const float si = fmaf(b2, s[i], (1.f - b2) * gi * gi);
  m[i] = mi;
  s[i] = si;
  // theta -= lr * m_hat / (sqrt(s_hat) + eps), with both bias corrections folded
  // into lr_t = lr * sqrt(1 - b2^t) / (1 - b1^t) and eps_t = eps * sqrt(1 - b2^t).
  theta[i] -= lr_t * mi / (sqrtf(si) + eps_t);
}

int adam_update(float* theta, const double* grad, float* m, float* s, int64_t p,
                const inrct_adam* a, cudaStream_t st) {
  INRCT_REQUIRE(a->t >= 1, "Adam step index t must be >= 1");
  INRCT_REQUIRE(m && s, "Adam moments must not be NULL");
  const double bc1 = 1.0 - pow(a->beta1, (double)a->t);
  const double bc2 = 1.0 - pow(a->beta2, (double)a->t);
  const float lr_t = (float)(a->lr * sqrt(bc2) / bc1);
  const float eps_t = (float)(a->eps * sqrt(bc2));
  adam_kernel<<<ceil_div(p, 256), 256, 0, st>>>(theta, grad, m, s, p, (float)a->beta1,
                                                (float)a->beta2, lr_t, eps_t);
  INRCT_CHECK_LAUNCH("adam");
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
