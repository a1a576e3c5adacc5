// Internal interface of the MLP translation units (FP32 SIMT and BF16 tcgen05).
#pragma once
#include "common.cuh"

namespace inrct {

constexpr int kMaxLayers = 10;  // n_hidden + 1 <= kMaxLayers
constexpr int kMaxHashLevels = 16;
constexpr int kMaxHashInputs = 64;  // hash levels x features per level

// Network description with theta offsets, built on the host from inrct_mlp.
struct Net {
  int kind;      // INRCT_FFN_RELU / INRCT_SIREN / INRCT_HASH
  int d, F, W, L;  // input dim, Fourier features, width, nonlinear layers
  float omega0;
  const float* B;  // device F x d
  const float* B_host;  // optional host copy of B (NULL if not given)
  int K0;          // input width of layer 1 (2F, d, or hash levels x features)
  int64_t p;       // parameter count
  // hash encoding: levels, features per level, log2 of the table size, the level
  // resolutions, and the table parameters (theta[0, n_table) holds the tables)
  int hL, hF, hlog2T;
  int hres[kMaxHashLevels];
  int64_t n_table;
  int fov;  // the grid's field of view (listed points outside it carry no weight)
  int64_t offW[kMaxLayers], offb[kMaxLayers];  // layer l = 0..L (L is the output layer)
  int in_dim[kMaxLayers], out_dim[kMaxLayers];
};

int make_net(const inrct_mlp* mlp, const inrct_grid* grid, Net* net);

// Grid index k -> pixel-centre coordinate -1 + (k + 1/2) 2/N = (2k + 1 - N) / N, formed
// as one correctly rounded FP32 division of exact integers (the FP32 value nearest
// the true centre).
__device__ __forceinline__ float grid_coord(int64_t k, int N) {
  return __fdiv_rn((float)(2 * k + 1 - N), (float)N);
}

// Integer numerators m_a = 2 k_a + 1 - N of the pixel-centre coordinates x_a = m_a / N of grid
// point i (x fastest; m_2 = 0 in 2-D).  Exact, |m_a| < N <= 4096.
__device__ __forceinline__ void point_numerators(int64_t i, int N, int d, int* m) {
  int64_t ix, iy, iz;
  if ((uint64_t)i <= 0xffffffffull) {
    const uint32_t u = (uint32_t)i, n = (uint32_t)N;
    const uint32_t q = u / n, q2 = q / n;
    ix = u - q * n;
    iy = q - q2 * n;
    iz = q2;
  } else {
    ix = i % N;
    iy = (i / N) % N;
    iz = i / ((int64_t)N * N);
  }
  m[0] = (int)(2 * ix + 1 - N);
  m[1] = (int)(2 * iy + 1 - N);
  m[2] = d == 3 ? (int)(2 * iz + 1 - N) : 0;
}

// Error-free sum: a + b = s + e exactly (Knuth's two-sum, no ordering assumption).
__device__ __forceinline__ float two_sum(float a, float b, float* e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  *e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// Phase of a Fourier feature, B . x reduced modulo 1 to t in about [-1/2, 1/2], for the grid
// point with coordinate numerators m (x_a = m_a / N), accurate to about an FP32 ulp of t.
// With x_a = m_a / N the phase is (sum_a B_a m_a) / N: each product B_a m_a (m_a is an exact
// FP32 integer) is p + e exactly by an FMA, the products are added with error-free sums into a
// head s and a tail, the quotient by N is q = s / N (a product with the reciprocal inv_N) with
// the remainder s - q N formed exactly by an FMA (q is within a few ulp of s / N, so the
// remainder is a small multiple of ulp(q) and representable), and
// t = (q - rint q) + (remainder + tail) / N.  Forming B . x from rounded coordinates in FP32
// instead leaves an absolute phase error of about |B . x| 2^-24 (2e-6 at |B . x| = 30), which
// moves features by about 2 pi times that: enough to flip the ReLU masks of units within
// 1e-5 of their RMS of zero.
__device__ __forceinline__ float ffn_phase_exact(float b0, float b1, float b2, const int* m, int d, int N,
                                                 float inv_N) {
  const float m0 = (float)m[0], m1 = (float)m[1], m2 = (float)m[2];
  const float p0 = __fmul_rn(b0, m0), e0 = __fmaf_rn(b0, m0, -p0);
  const float p1 = __fmul_rn(b1, m1), e1 = __fmaf_rn(b1, m1, -p1);
  float t1;
  float s = two_sum(p0, p1, &t1);
  float tail = __fadd_rn(__fadd_rn(e0, e1), t1);
  if (d == 3) {
    const float p2 = __fmul_rn(b2, m2), e2 = __fmaf_rn(b2, m2, -p2);
    float t2;
    s = two_sum(s, p2, &t2);
    tail = __fadd_rn(tail, __fadd_rn(e2, t2));
  }
  const float fN = (float)N;
  const float q = __fmul_rn(s, inv_N);
  const float r = __fmaf_rn(-q, fN, s);  // s - q N, exact
  const float t = __fsub_rn(q, rintf(q));
  return __fmaf_rn(__fadd_rn(r, tail), inv_N, t);
}

// sin(2 pi t) and cos(2 pi t) for |t| <= 1/2 + a few ulp, to about 1e-7 absolute.  The angle is
// reduced to the nearest quarter turn k / 4 (exactly: r = t - k/4 by Sterbenz's lemma), so that
// x = 2 pi r lies in [-pi/4, pi/4]; 2 pi is taken as a two-term FP32 sum.  There the Taylor
// series of sin to x^9 and of cos to x^10 are within 2e-9 of the functions (the first omitted
// terms, x^11/11! and x^12/12!, at x = pi/4), evaluated by Horner's rule in FP32; the quarter
// turn then rotates (sin, cos) by k pi / 2.  About twenty FP32 instructions, no branch.
__device__ __forceinline__ void sincos_turns(float t, float* s, float* c) {
  const float k = rintf(4.f * t);
  const float r = __fmaf_rn(-0.25f, k, t);
  const float kTwoPiHi = 6.28318548202514648f;        // fl(2 pi)
  const float kTwoPiLo = -1.74845553146951715e-07f;   // 2 pi - fl(2 pi)
  const float x = __fmaf_rn(r, kTwoPiHi, __fmul_rn(r, kTwoPiLo));
  const float x2 = __fmul_rn(x, x);
  float ps = __fmaf_rn(x2, 1.f / 362880.f, -1.f / 5040.f);
  ps = __fmaf_rn(x2, ps, 1.f / 120.f);
  ps = __fmaf_rn(x2, ps, -1.f / 6.f);
  const float sn = __fmaf_rn(__fmul_rn(x2, ps), x, x);
  float pc = __fmaf_rn(x2, -1.f / 3628800.f, 1.f / 40320.f);
  pc = __fmaf_rn(x2, pc, -1.f / 720.f);
  pc = __fmaf_rn(x2, pc, 1.f / 24.f);
  pc = __fmaf_rn(x2, pc, -0.5f);
  const float cs = __fmaf_rn(x2, pc, 1.f);
  const int q = ((int)k) & 3;
  const float a = (q & 1) ? cs : sn, b = (q & 1) ? sn : cs;  // (sin, cos) of r rotated by q quarter turns
  *s = (q == 1 || q == 0) ? a : -a;
  *c = (q == 0 || q == 3) ? b : -b;
}

// Coordinates of grid point i (x fastest).  Indices below 2^32 take 32-bit divisions (the
// 64-bit ones are a long instruction sequence, on the path of every tile's set-up).
__device__ __forceinline__ void point_coords(int64_t i, int N, int d, float* x) {
  int64_t ix, iy, iz;
  if ((uint64_t)i <= 0xffffffffull) {
    const uint32_t u = (uint32_t)i, n = (uint32_t)N;
    const uint32_t q = u / n, q2 = q / n;
    ix = u - q * n;
    iy = q - q2 * n;
    iz = q2;
  } else {
    ix = i % N;
    iy = (i / N) % N;
    iz = i / ((int64_t)N * N);
  }
  x[0] = grid_coord(ix, N);
  x[1] = grid_coord(iy, N);
  x[2] = d == 3 ? grid_coord(iz, N) : 0.f;
}

// FP32 SIMT path
size_t simt_eval_ws_bytes(const Net& net);
int simt_eval(const Net& net, const float* theta, int N, int64_t n, float* image, void* ws,
              size_t ws_bytes, cudaStream_t st);
size_t simt_vjp_ws_bytes(const Net& net, int64_t n_idx);
int simt_vjp(const Net& net, const float* theta, int N, const int32_t* idx, int64_t n_idx,
             const float* v, double scale, double* grad_f64, float* grad_f32, double* value_out,
             void* ws, size_t ws_bytes, cudaStream_t st);

// BF16 tcgen05 path
bool tc_supported(const Net& net, char* why, size_t why_len);
// BF16 weights prepared once (grad_step shares them between evaluation and VJP);
// `prepared` may be NULL, then each call converts theta itself.
size_t tc_weights_bytes(const Net& net);
int tc_prepare(const Net& net, const float* theta, void* buf, size_t bytes, cudaStream_t st);
size_t tc_eval_ws_bytes(const Net& net);
int tc_eval(const Net& net, const float* theta, int N, int64_t n, float* image, void* ws,
            size_t ws_bytes, cudaStream_t st, const void* prepared = nullptr);
size_t tc_vjp_ws_bytes(const Net& net, int64_t n_idx);
// value_out (nullable): the virtual loss scale * sum v_i f(x_i) of Eq. 3, FP64 device scalar.
int tc_vjp(const Net& net, const float* theta, int N, const int32_t* idx, int64_t n_idx,
           const float* v, double scale, double* grad_f64, float* grad_f32, double* value_out,
           void* ws, size_t ws_bytes, cudaStream_t st, const void* prepared = nullptr);
// Reads and clears the bounded-wait status word of the current device after synchronising
// st; *code = 0 when no wait gave up since the last read.
int tc_device_status(cudaStream_t st, int* code);
// Looks up the status word's address on the current device (before a stream capture).
int tc_status_resolve(cudaStream_t st);
// Limit of every bounded wait of later launches (0: the default, 1 s).
void tc_set_wait_limit(unsigned long long ns);
// Test hook: while on, the tile kernel's producer issues no weight loads.
void tc_set_stall_loads(int on);

// split-K TN GEMM of the weight gradients, exposed for diagnostics
size_t gemm_tn_ws_bytes(int64_t K, int M, int N);
// sin(pi x), cos(pi x) by the tile kernel's feature polynomial, for diagnostics.
int sincospi_diag(const float* x, float* s, float* c, int64_t n, cudaStream_t st);
int gemm_tn(const void* X, const void* Y, const void* Y16, int64_t K, int M, int N, float* C, void* ws,
            size_t ws_bytes, cudaStream_t st);

// shared small kernels (optim.cu)
int adam_update(float* theta, const double* grad, float* m, float* s, int64_t p,
                const inrct_adam* adam, cudaStream_t st);
// Adam reading the step index from *t_dev (device); a->t is ignored.
int adam_update_devt(float* theta, const double* grad, float* m, float* s, int64_t p,
                     const inrct_adam* a, const long long* t_dev, cudaStream_t st);
// *t_dev += 1 on the stream.
int advance_step_counter(long long* t_dev, cudaStream_t st);
int f64_to_f32(const double* in, float* out, int64_t n, cudaStream_t st);
// image[i] = 0 for the grid points outside the field of view.
int fov_zero(float* image, int64_t n, int N, cudaStream_t st);
size_t check_index_ws_bytes(int64_t n);
int check_index_set(const int32_t* idx, int64_t n_idx, int64_t n, int N, int fov, void* ws, size_t ws_bytes,
                    long long* counts_out, cudaStream_t st);

// Points processed per VJP chunk: scratch is sized for min(n_idx, this).
constexpr int64_t kVjpChunk = int64_t(1) << 20;

}  // namespace inrct
