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
