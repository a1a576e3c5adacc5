// BF16 tensor-core (tcgen05) path of the INR: grid evaluation E{f} (Sec. 3)
// and the residual-weighted VJP of Eq. (2) / the virtual loss of Eq. (3).
//
// Fused MLP tile engine (mlp_tile_kernel)
// ---------------------------------------
// A persistent CTA (one per SM) walks tiles of 128 points, two at a time (slots 0
// and 1).  Per tile it runs a program of GEMM stages, each
// D[128 x W] = A[128 x K] * B[W x K]^T with A the stage input (BF16, in shared
// memory, K-major 64-column panels) and B a weight matrix streamed by TMA through
// a 64 KB ring of 64-column chunks; D accumulates in FP32 in tensor memory, one
// W-column accumulator per slot, so the tensor core works on one slot while the
// epilogue drains the other.  Warp roles (18 warps):
//   warps 0-15  epilogue: build the first input (Fourier features or the SIREN
//               first layer, FP32 on the CUDA cores), then after every stage read
//               D from TMEM, add the bias, apply the activation (FP32) and write
//               the next stage's BF16 A panels; the small parameter tables are
//               staged in shared memory.
//   warp 16     TMA producer of the weight ring.
//   warp 17     MMA issuer (one thread).
// SIREN layers keep omega0 folded into their BF16 weights and FP32 biases
// (u = omega0 (W h + b) = W' h + b'), so the epilogue applies sin(u).
//
// VJP program: the forward stages, then backward stages
// delta_{l-1} = (W'_l^T delta_l) * sigma'(u_{l-1}) fed by a transposed weight
// copy.  The epilogues write, for the listed points only, the activations a_l,
// the deltas delta_l (and cos(u_l) for SIREN) to scratch, [points][features]
// BF16.  A split-K TN GEMM (tn_gemm_kernel) then forms
// dW_l = sum_points delta_l a_{l-1}^T and db_l = sum_points delta_l (a ones
// operand) with MN-major operands straight from that scratch; FP32 partials
// per split are reduced in FP64 into the gradient.  Scratch grows with the
// number of listed points (chunked), never with the grid.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <type_traits>

#include "mlp.cuh"
#include "tc_ptx.cuh"

namespace inrct {

using namespace tc;

namespace {

constexpr int kTile = 128;       // points per tile (MMA M)
constexpr int kNSplit = 1;       // MMA N-groups per weight K-panel: N = W / kNSplit
constexpr int kKChunk = 64;      // K per weight ring slot (16, 32 or 64: 32-, 64-, 128-byte swizzle);
                                 // 64 measured fastest: each slot costs a fixed hand-off
// Weight ring: ring_bytes(mode) / (W / kNSplit * 2 kKChunk B) slots.  64 KB in both modes: the
// weights arrive ahead of the MMAs with two slots (loading each slot only once changes the
// evaluation's time by 1 %), and the room a deeper ring would take holds the staged parameter
// tables instead.
__host__ __device__ constexpr int ring_bytes(int) { return 64 * 1024; }
constexpr int kRingMax = 8;
// 64-bit words after the ring: 2 kRingMax + 31 barriers, then tmem base and abort flag (one word)
constexpr int kTileBars = 2 * kRingMax + 31 + 1;
constexpr int kPanelBytes = kTile * 128;  // one 64-column BF16 panel of 128 rows
constexpr int kMaxStages = 2 * kMaxLayers;
constexpr int kMaxJobs = 24;
constexpr int kMaxSplits = 16;   // split-K factor of the weight-gradient GEMM

// FFN input columns are interleaved per 64-column panel: panel c holds cos(2 pi B_f x) for
// f = 32c .. 32c+31 in its first 32 columns and sin(2 pi B_f x) of the same features in the
// last 32, so that one sincospif gives both entries of a feature.  ffn_orig_col maps a
// panel column back to the input column of gamma(x) = [cos 2 pi B x; sin 2 pi B x].
__host__ __device__ inline int ffn_orig_col(int kp, int F) {
  const int c = kp >> 6, j = kp & 63;
  return j < 32 ? 32 * c + j : F + 32 * c + (j - 32);
}
__host__ __device__ inline int ffn_panel_col(int k, int F) {
  return k < F ? 64 * (k >> 5) + (k & 31) : 64 * ((k - F) >> 5) + 32 + ((k - F) & 31);
}


// ---------------------------------------------------------------------------
// Status of the bounded waits.  Every mbarrier wait of the tensor-core kernels gives up after
// a limit; the first wait that does records its code here (one word per device, read and
// cleared by inrct_device_status): 1xx weight-gradient GEMM, 2xx weight producer, 3xx MMA
// issuer, 4xx epilogue; 901 shared memory not 1024-byte aligned.
// ---------------------------------------------------------------------------
__device__ int g_wait_status;

std::atomic<unsigned long long> g_wait_ns{kWaitTimeoutNs};
std::atomic<int> g_stall_loads{0};
std::mutex g_status_mu;
void* g_status_addr[256] = {};

// Device address of the status word on the current device: looked up with
// cudaGetSymbolAddress on every call outside stream capture (cheap, and never stale after a
// device reset), taken from the per-device cache during capture.
int status_word(cudaStream_t st, int** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) {
    set_error("no usable current device (%s)", cudaGetErrorString(e));
    return INRCT_ERR_CUDA;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturing = st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
  std::lock_guard<std::mutex> lk(g_status_mu);
  if (!capturing || !g_status_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_wait_status);
    if (e != cudaSuccess || !p) {
      set_error("status word: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return INRCT_ERR_CUDA;
    }
    g_status_addr[dev] = p;
  }
  *out = static_cast<int*>(g_status_addr[dev]);
  return INRCT_OK;
}

// ---------------------------------------------------------------------------
// host: tensor maps
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D BF16 row-major tensor [outer][inner], 128-byte swizzled boxes of {box_inner, box_outer}.
int make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
             uint32_t box_outer, int swizzle_bytes = 128) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is unavailable from the driver");
    return INRCT_ERR_CUDA;
  }
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                       : (swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B),
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d): dims %llu x %llu box %u x %u", (int)r,
              (unsigned long long)inner, (unsigned long long)outer, box_inner, box_outer);
    return INRCT_ERR_CUDA;
  }
  return INRCT_OK;
}

struct Maps {
  CUtensorMap m[kMaxJobs];
};

// Launch-parameter copy of the first-layer table of a Fourier-feature network (entries
// {B_0, B_1, B_2, 0} as in PrepTable), for the grid evaluation: read through the constant
// cache, it takes nothing from the shared-memory bandwidth the MMAs' operand reads use.  n = 0:
// not given (the kernel reads the table from shared memory).  Other kernel instances take the
// 4-byte placeholder.
constexpr int kMaxConstFirst = 1024;
struct FirstConst {
  int n;
  float4 c[kMaxConstFirst];
};
struct NoFirstConst {
  int n;
};
template <int MODE, int KIND, bool SPLIT>
struct FirstArg {
  using type = NoFirstConst;
};
template <>
struct FirstArg<0, INRCT_FFN_RELU, false> {
  using type = FirstConst;
};

// ---------------------------------------------------------------------------
// weight preparation: BF16 (W' = scale W) row-major and transposed, FP32 biases
// ---------------------------------------------------------------------------
struct PrepTable {
  int n;
  int out[kMaxLayers], in[kMaxLayers];
  int64_t offW[kMaxLayers], offb[kMaxLayers];
  __nv_bfloat16* Wb[kMaxLayers];
  __nv_bfloat16* WbT[kMaxLayers];
  __nv_bfloat16* Wlo[kMaxLayers];  // split forward stages: bf16(W' - Wb), else NULL
  float* bias[kMaxLayers];
  int permF;  // FFN: F, and entry 0 (layer 0) is stored with interleaved input columns; else 0
  // the row blockIdx.y == n fills the small tables the tile kernel reads through L1:
  // first-layer table (SIREN {w'_0, w'_1, w'_2, b'} per output; FFN {B_0, B_1, B_2, 0} per
  // feature) and an aligned copy of the output-layer weights
  int kind, d, n_first, W;
  int64_t offW0, offb0, offWout;
  const float* B;
  float4* first;
  float* wout;
};

// All MMA layers in one launch: blockIdx.y selects the layer.
__global__ void prep_all_kernel(const float* __restrict__ theta, const __grid_constant__ PrepTable T,
                                float scale) {
  const int l = blockIdx.y;
  if (l == T.n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.n_first; i += gridDim.x * blockDim.x) {
      if (T.kind == INRCT_SIREN) {
        const float* w1 = theta + T.offW0 + (int64_t)i * T.d;
        T.first[i] = make_float4(scale * w1[0], scale * w1[1], T.d == 3 ? scale * w1[2] : 0.f,
                                 scale * theta[T.offb0 + i]);
      } else {
        const float* bf = T.B + (int64_t)i * T.d;
        T.first[i] = make_float4(bf[0], bf[1], T.d == 3 ? bf[2] : 0.f, 0.f);
      }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.W; i += gridDim.x * blockDim.x)
      T.wout[i] = theta[T.offWout + i];
    return;
  }
  const int out = T.out[l], in = T.in[l];
  const int64_t cnt = (int64_t)out * in;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int o = (int)(t / in), k = (int)(t % in);
    const float wf = scale * theta[T.offW[l] + t];
    const __nv_bfloat16 w = __float2bfloat16_rn(wf);
    const int kw = (l == 0 && T.permF > 0) ? ffn_panel_col(k, T.permF) : k;
    T.Wb[l][(int64_t)o * in + kw] = w;
    if (T.WbT[l]) T.WbT[l][(int64_t)kw * out + o] = w;
    if (T.Wlo[l]) T.Wlo[l][(int64_t)o * in + kw] = __float2bfloat16_rn(wf - __bfloat162float(w));
    if (t < out) T.bias[l][t] = scale * theta[T.offb[l] + t];
  }
}

// ---------------------------------------------------------------------------
// split-K TN GEMM:  C[m][n] = sum_k X[k][m] * Y[k][n]   (X, Y BF16, MN-major)
// plus two optional 16-column blocks: ones (C1[m] = sum_k X[k][m]) and a
// K-major [16][K] operand Y16 (C2[m][c] = sum_k X[k][m] Y16[c][k]).
// Output: FP32 partial per split, [split][M][ldc] with ldc = N + 32.
// ---------------------------------------------------------------------------
struct GemmJob {
  int M, N, n0;           // rows (multiple of 128), main columns (0 or multiple of 64, <= 256), Y column offset
  int has_ones, has_y16;  // extra column blocks
  int mx, my, my16;       // map indices
  int mtiles;             // M / 128
  int64_t part_off;       // offset (floats) of this job's partials
  // reduction into theta's gradient
  int64_t offW;  // gradient offset of the weight block (row stride ldW)
  int ldW;       // row length of the weight block in theta
  int w_src;     // 0: main columns [0, w_cols); 1: y16 columns [0, w_cols)
  int w_cols;
  int64_t offb;  // gradient offset of the bias (or -1)
  double mult;   // omega0 for SIREN sine layers, else 1
  int permF;     // FFN layer 0: main columns are interleaved panel columns of F features
};

struct GemmPlan {
  int n_jobs;
  int S;              // splits of K
  int64_t K;          // points
  int64_t per_split;  // points per split (multiple of 64)
  int cta_begin[kMaxJobs + 1];
  GemmJob job[kMaxJobs];
  // output-layer bias gradient: FP64 partial sums of scale * v_i from the VJP tile kernel,
  // summed by the reduction's extra block row into grad[off_bout] (n_bpart == 0: none)
  const double* bpart;
  int n_bpart;
  int64_t off_bout;
  // the virtual loss (Eq. 3): FP64 partial sums of scale * v_i * f(x_i) from the VJP tile
  // kernel (n_bpart of them), summed by the same block into *value_out (NULL: not wanted)
  const double* vpart;
  double* value_out;
  uint64_t wait_ns;  // limit of every bounded wait of the GEMM kernel
};

constexpr int kGemmStages = 4;
constexpr int kGemmStageBytes = 16384 + 32768 + 2048;  // X (128 x 64), Y (64 x 256), Y16 (16 x 64)

__global__ void __launch_bounds__(192, 1)
    tn_gemm_kernel(const __grid_constant__ Maps maps, const __grid_constant__ GemmPlan plan,
                   float* __restrict__ part,
                   int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  uint8_t* ones = smem + kGemmStages * kGemmStageBytes;  // 16 rows x 128 B of BF16 ones
  __shared__ uint64_t full[kGemmStages], empty[kGemmStages], accf;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  int jb = 0;
  while (jb + 1 < plan.n_jobs && (int)blockIdx.x >= plan.cta_begin[jb + 1]) ++jb;
  const GemmJob& J = plan.job[jb];
  const int local = blockIdx.x - plan.cta_begin[jb];
  const int mt = local % J.mtiles, sp = local / J.mtiles;
  const int64_t k_begin = (int64_t)sp * plan.per_split;
  const int64_t k_end = min(plan.K, k_begin + plan.per_split);
  const int nch = k_end > k_begin ? (int)((k_end - k_begin + 63) / 64) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGemmStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accf, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < 16 * 128 / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(ones)[i] = 0x3F803F80u;  // two BF16 ones
  fence_async_smem();
  if (warp == 2) tmem_alloc(&tmem_base, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t xbytes = 2 * 8192, ybytes = (uint32_t)J.N * 128, y16bytes = J.has_y16 ? 2048 : 0;

  const uint64_t lim = plan.wait_ns;
  if (warp == 0) {
    if (lane == 0) {
      uint32_t ep = 1;
      int armed = 0;  // loads issued
      for (int c = 0; c < nch; ++c) {
        const int s = c % kGemmStages;
        if (c > 0 && s == 0) ep ^= 1;
        if (!mbar_wait(&empty[s], ep, &abort_flag, err, 101, lim)) break;
        uint8_t* st = smem + s * kGemmStageBytes;
        mbar_arrive_expect_tx(&full[s], xbytes + ybytes + y16bytes);
        const int k0 = (int)(k_begin + 64 * c);
        tma_load_2d(st, &maps.m[J.mx], &full[s], mt * 128, k0);
        tma_load_2d(st + 8192, &maps.m[J.mx], &full[s], mt * 128 + 64, k0);
        for (int b = 0; b < J.N / 64; ++b)
          tma_load_2d(st + 16384 + b * 8192, &maps.m[J.my], &full[s], J.n0 + 64 * b, k0);
        if (J.has_y16) tma_load_2d(st + 16384 + 32768, &maps.m[J.my16], &full[s], k0, 0);
        ++armed;
      }
      // no load may still be writing shared memory when the CTA exits (the abort path leaves
      // loads the MMA thread never waited for): wait for the last stages' loads to land
      for (int c = armed > kGemmStages ? armed - kGemmStages : 0; c < armed; ++c)
        mbar_wait_drain(&full[c % kGemmStages], (uint32_t)((c / kGemmStages) & 1), lim);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t fp = 0;
      const uint32_t id_main = idesc_bf16(128, J.N > 0 ? J.N : 16, true, true);
      const uint32_t id_16 = idesc_bf16(128, 16, true, false);
      bool issued = false;
      for (int c = 0; c < nch; ++c) {
        const int s = c % kGemmStages;
        if (c > 0 && s == 0) fp ^= 1;
        if (!mbar_wait(&full[s], fp, &abort_flag, err, 102, lim)) break;
        tc_fence_after();
        const uint32_t st = smem_u32(smem + s * kGemmStageBytes);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint64_t ad = desc_sw128(st + j * 2048, 8192, 1024);
          const uint32_t acc = (c > 0 || j > 0) ? 1u : 0u;
          if (J.N > 0) mma_bf16(tmem, ad, desc_sw128(st + 16384 + j * 2048, 8192, 1024), id_main, acc);
          if (J.has_ones) mma_bf16(tmem + 256, ad, desc_sw128(smem_u32(ones) + j * 32, 16, 1024), id_16, acc);
          if (J.has_y16)
            mma_bf16(tmem + 272, ad, desc_sw128(st + 16384 + 32768 + j * 32, 16, 1024), id_16, acc);
        }
        issued = true;
        mma_commit(&empty[s]);
      }
      if (issued) {
        mma_commit(&accf);
        // every issued MMA completes before the tensor memory is released (on the abort path
        // the epilogue does not wait for them)
        mbar_wait_drain(&accf, 0, lim);
      } else {
        mbar_arrive(&accf);
      }
    }
  } else {
    // epilogue warps 2..5: lanes 32*(warp%4) .. of TMEM = rows of C
    const int q = warp & 3;
    const int row = mt * 128 + q * 32 + lane;
    const int ldc = J.N + 32;
    float* out = part + J.part_off + ((int64_t)sp * J.M + row) * ldc;
    const bool ok = warp_wait(&accf, 0, &abort_flag, err, 103, lim);
    tc_fence_after();
    float v[32];
    auto emit = [&](int col, int tcol) {
      if (nch > 0 && ok) {
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + tcol, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *reinterpret_cast<float4*>(out + col + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    };
    for (int c0 = 0; c0 < J.N; c0 += 32) emit(c0, c0);
    // ones block (16 columns) and the Y16 block (16 columns); absent blocks hold zeros
    if (nch > 0 && ok) {
      tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + 256, v);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if (!J.has_ones) v[i] = 0.f;
      if (!J.has_y16) v[16 + i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < 32; i += 4)
      *reinterpret_cast<float4*>(out + J.N + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// grad[...] (+)= mult * sum_s part[s][m][c] for every (job, m, c) that maps to theta.
__global__ void gemm_reduce_kernel(const __grid_constant__ GemmPlan plan, const float* __restrict__ part,
                                   int accumulate, double* __restrict__ grad) {
  const int jb = blockIdx.y;
  if (jb == plan.n_jobs) {  // output bias and virtual loss: fixed-order trees over the partials
    if (blockIdx.x != 0) return;
    __shared__ double sh[256];
    for (int which = 0; which < 2; ++which) {
      const double* src = which ? plan.vpart : plan.bpart;
      if (which && !plan.value_out) break;
      double s = 0.0;
      for (int i = threadIdx.x; i < plan.n_bpart; i += blockDim.x) s += src[i];
      sh[threadIdx.x] = s;
      __syncthreads();
      for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        double* dst = which ? plan.value_out : grad + plan.off_bout;
        *dst = accumulate ? *dst + sh[0] : sh[0];
      }
      __syncthreads();
    }
    return;
  }
  const GemmJob& J = plan.job[jb];
  const int cols = J.w_cols + (J.offb >= 0 ? 1 : 0);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)J.M * cols) return;
  const int m = (int)(e / cols), c = (int)(e % cols);
  const int ldc = J.N + 32;
  int col;
  int64_t dst;
  if (c < J.w_cols) {
    col = J.w_src == 0 ? c : J.N + 16 + c;
    const int kc = J.permF > 0 ? ffn_orig_col(J.n0 + c, J.permF) : J.n0 + c;
    dst = J.offW + (int64_t)m * J.ldW + kc;
  } else {
    col = J.N;  // first column of the ones block
    dst = J.offb + m;
  }
  // all split partials are loaded before the in-order FP64 sum (independent loads in flight)
  float pv[kMaxSplits];
#pragma unroll
  for (int q = 0; q < kMaxSplits; ++q)
    pv[q] = q < plan.S ? part[J.part_off + ((int64_t)q * J.M + m) * ldc + col] : 0.f;
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kMaxSplits; ++q)
    if (q < plan.S) s += (double)pv[q];
  s *= J.mult;
  grad[dst] = accumulate ? grad[dst] + s : s;
}


// ---------------------------------------------------------------------------
// fused MLP tile engine
// ---------------------------------------------------------------------------
enum StageKind { kFwdHidden = 0, kFwdLast = 1, kBwd = 2 };

struct TileProg {
  int mode;  // 0 eval, 1 vjp
  int kind, d, F, W, L, N;
  int64_t n_grid, npts;
  int fov;  // VJP: listed points outside the grid's field of view carry no weight
  float omega0;
  const float* B;       // F x d (FFN)
  const float* theta;   // FP32 parameters (SIREN first layer, output layer)
  const float* bias;    // folded FP32 biases, [L][W]
  const float4* first;  // first-layer table (see PrepTable)
  int n_first;          // its entries (SIREN W, FFN F)
  int first_staged;     // the table fits the shared-memory staging area
  const float* wout;    // output-layer weights [W], 16-byte aligned
  int64_t offW0, offb0, offWout, offbout;  // theta offsets (first layer, output layer)
  int n_stages;
  int st_kind[kMaxStages], st_layer[kMaxStages], st_panels[kMaxStages], st_map[kMaxStages];
  int st_map_lo[kMaxStages];  // split forward stages: map of the low parts W_lo of the weights
  int in_panels;        // panels of the first stage's input
  // eval
  float* out;
  // vjp
  const int32_t* idx;
  const float* v;
  float scale;
  __nv_bfloat16* E;     // [npts_pad][2F] layer-1 input (FFN)
  __nv_bfloat16* Act;   // [L][npts_pad][W] activations a_l; a_0 .. a_{L-2} arrive by TMA store
  __nv_bfloat16* Dlt;   // [L][npts_pad][W] deltas, all by TMA store from the input panels
  // sigma'(u_l) for l = 0 .. L-2 of the SIREN (cos u_l with omega0 folded in the weights; the split
  // VJP of ReLU networks keeps its masks as bits instead), read back only by this kernel:
  // blocked so that a warp's 32 rows x CW columns are one
  // contiguous 1 KB run, index (((l * n_tiles + tile) * W/64 + c) * NWG + g) * 128 + row
  __nv_bfloat16* Sg;
  int st_in_arr[kMaxStages];    // the stage's input panels are row block tile of: 0 Act, 1 Dlt, -1 none
  int st_in_layer[kMaxStages];  // ... layer of that array
  int tail_layer;               // Dlt layer held by the panels after the last stage
  int map_act, map_dlt;         // tensor maps (in the kernel's Maps) for the panel stores
  // 16-row K-major GEMM operands; only rows 0..2 of Y16c (coordinates, SIREN; row d.. zero for
  // d = 2) and row 0 of Y16o (scale * v) are written: the other rows only feed output columns
  // of the weight-gradient GEMM that the reduction never reads (each column depends on its row)
  __nv_bfloat16* Y16c;  // [16][npts_pad]
  __nv_bfloat16* Y16o;  // [16][npts_pad]
  double* bias_part;    // [gridDim.x][4] FP64 sums of scale * v_i (output-layer bias gradient)
  double* vloss_part;   // [gridDim.x][4] FP64 sums of scale * v_i * f(x_i) (the virtual loss, Eq. 3)
  int64_t npts_pad;
  int stall;            // test hook: the producer issues no weight loads (a bounded wait runs out)
  uint64_t wait_ns;     // limit of every bounded wait
};

template <int CW>
__device__ __forceinline__ void store_row_bf16(__nv_bfloat16* dst, const float* v) {
  uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int q = 0; q < CW / 8; ++q)
    d4[q] = make_uint4(pack_bf16(v[8 * q], v[8 * q + 1]), pack_bf16(v[8 * q + 2], v[8 * q + 3]),
                       pack_bf16(v[8 * q + 4], v[8 * q + 5]), pack_bf16(v[8 * q + 6], v[8 * q + 7]));
}

template <int CW>
__device__ __forceinline__ void load_row_bf16(const __nv_bfloat16* src, float* v) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
  for (int q = 0; q < CW / 8; ++q) {
    const uint4 w = s4[q];
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[8 * q + 2 * k] = __uint_as_float(u[k] << 16);
      v[8 * q + 2 * k + 1] = __uint_as_float(u[k] & 0xffff0000u);
    }
  }
}

// Fourier feature of phase ph: cos or sin of 2 pi ph.  ph is reduced to t = ph - rint(ph)
// in [-1/2, 1/2] exactly, then sincospif(2t) (accurate to about an FP32 ulp).  The features
// feed ReLU mask decisions downstream, so they are computed accurately rather than with the
// hardware approximations (those, 2^-21.4 absolute, moved the BF16 gradient of a 3-D FFN by
// more than 1 % through flipped masks; measured).
// Features of the VJP, whose ReLU masks downstream must be decided at FP32 accuracy: sin and
// cos of 2 pi t to about 1e-7 (sincos_turns).
__device__ __forceinline__ void feat_sincos(float t, float* s, float* c) { sincos_turns(t, s, c); }
// Grid evaluation: the features only enter BF16 operands (rounded to about 4e-3 relative) and
// decide no mask that a gradient uses, so after the same exact reduction to [-1/2, 1/2] the
// hardware sine and cosine of 2 pi t (about 2^-21 absolute on [-pi, pi]) are accurate enough
// and cost one special-function instruction each instead of a range-reduced polynomial.
__device__ __forceinline__ void four_feat_fast(float ph, float* s, float* c) {
  __sincosf(6.28318530717958647692f * __fsub_rn(ph, rintf(ph)), s, c);
}


// Two tiles are in flight per CTA (slots 0 and 1), each with one FP32 accumulator of
// W TMEM columns and its own four input panels.  The MMA issuer alternates the slots
// stage by stage, (slot 0, stage s), (slot 1, stage s), (slot 0, stage s+1), ..., so
// that while the epilogue works on one slot the tensor core works on the other.
// Weights go through a ring of chunks of NW = W / kNSplit rows x 64 K (128B swizzle);
// each K-panel of a stage is kNSplit MMA groups of N = NW.  N = W = 256 runs the tensor
// core at its peak; N = 128 needs twice the MMA instructions from the single issuing
// thread and falls behind when the epilogue warps keep its SMSP busy.
//
// Hand-off per slot and stage: the epilogue waits for acc_full[t] (every MMA of the
// stage has completed, so the slot's input panels are free as well), reads the
// accumulator, writes the next stage's input panels and arrives once per warp on
// in_ready[t], which the MMA issuer waits for before the slot's next stage: one
// arrival means both "accumulator drained" and "next input written".  Only the
// first stage may have more than four input panels (Fourier features, 2F > 256);
// those are streamed through the four panel buffers with per-panel barriers
// (a_full: written, a_empty: read by the MMA).
//
// SPLIT (the VJP of ReLU networks).  The forward stages decide the ReLU masks that the
// backward stages apply, and a mask decided on BF16-rounded operands differs from the
// exact one wherever a pre-activation lies within BF16 rounding of zero (about 1 % of the
// units of the 3-D Fourier-feature networks, several per point).  So the forward stages
// form their pre-activations to about FP32 accuracy: every operand x is split into
// x_hi = bf16(x) and x_lo = bf16(x - x_hi), and the stage accumulates
// a_hi W_hi^T + a_lo W_hi^T + a_hi W_lo^T in FP32 (the dropped a_lo W_lo^T and the
// rounding of the low parts are about 2^-16 of each product).  The low parts of a stage's
// input take the panel space of the second slot, so one tile is in flight per CTA
// (NSLOT = 1); the ring carries the W_hi and W_lo chunks of each K panel in turn.  The
// backward stages and the scratch the weight-gradient GEMM reads stay single BF16.
//
// NWG epilogue warpgroups; each thread of warpgroup g owns CW = 64/NWG columns of
// every 64-column chunk of its TMEM lane (row).
template <int MODE, int KIND, int NWG, bool SPLIT>
__global__ void __launch_bounds__(32 * (4 * NWG + 2), 1)
    mlp_tile_kernel(const __grid_constant__ Maps maps, const __grid_constant__ TileProg P,
                    const __grid_constant__ typename FirstArg<MODE, KIND, SPLIT>::type FC,
                    int* __restrict__ err) {
  constexpr int NSLOT = SPLIT ? 1 : 2;
  static_assert(!SPLIT || MODE == 1, "split operands serve the VJP's mask decisions");
  // Grid evaluation of a Fourier-feature network: the first stage of the two slots runs jointly.
  // The epilogue writes feature panel c of both tiles from one read of the features'
  // coefficients, and the MMA issuer applies each weight chunk of that stage to both tiles.
  constexpr bool kJoint0 = MODE == 0 && KIND == INRCT_FFN_RELU && NSLOT == 2;
  // Dynamic shared memory only (no static): [8 input panels][weight ring][barriers][dot scratch].
  // The panels and the ring need 1024-byte alignment (128-byte swizzle atoms); the dynamic
  // window starts there when the kernel has no static shared memory, which is checked.
  extern __shared__ __align__(1024) uint8_t dsm[];
  if ((smem_u32(dsm) & 1023u) != 0) {
    if (threadIdx.x == 0) atomicCAS(err, 0, 901);
    return;
  }
  uint8_t* smem = dsm;
  const int W = P.W;
  const int NW = W / kNSplit;                    // MMA N and weight rows per ring slot
  uint8_t* apan = smem;                          // 2 slots x 4 x 16 KB input panels (SPLIT: hi, lo)
  uint8_t* ring = smem + 8 * kPanelBytes;        // n_ring x (NW x 2 kKChunk B) weight chunks
  const uint32_t chunk_bytes = (uint32_t)NW * (2 * kKChunk);
  const int n_ring = ring_bytes(MODE) / (int)chunk_bytes;
  constexpr int CW = 64 / NWG, EPI_WARPS = 4 * NWG;  // one arrival per epilogue warp
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring + ring_bytes(MODE));
  uint64_t* w_full = bars;                       // [kRingMax]
  uint64_t* w_empty = w_full + kRingMax;         // [kRingMax]
  uint64_t* in_ready = w_empty + kRingMax;       // [2]
  uint64_t* acc_full = in_ready + 2;             // [2]
  uint64_t* a_full = acc_full + 2;               // [2][4]
  uint64_t* a_empty = a_full + 8;                // [2][4]
  uint64_t* dot_bar = a_empty + 8;               // [4] per row quarter: partial dots written
  uint64_t* dot_free = dot_bar + 4;              // [4]: the summing warp has read them
  uint64_t* st_done = dot_free + 4;              // [2]
  uint64_t* drain_bar = st_done + 2;
  uint32_t* tmem_base = reinterpret_cast<uint32_t*>(drain_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_base + 1);
  float* dotp = reinterpret_cast<float*>(bars + kTileBars);  // [NWG][kTile]
  // The small parameter tables are staged in shared memory after the dot scratch.  All lanes
  // of a warp read the same entry: from shared memory that is a broadcast, while through L1
  // each such load returned a copy per lane (evaluation of 512^2 points of the SIREN 5 x 256:
  // 179 -> 169 us, together with the paired accumulator loads below).
  float* bias_s = dotp + NWG * kTile;                   // [L][W]
  float* wout_s = bias_s + (size_t)P.L * W;             // [W]
  float4* first_s = reinterpret_cast<float4*>(wout_s + W);  // [n_first] when P.first_staged
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t lim = P.wait_ns;
  const int64_t n_tiles = (P.npts + kTile - 1) / kTile;
  // this CTA's tiles are blockIdx.x + j * gridDim.x; they are taken in groups of NSLOT
  // (slot 0, slot 1)
  const int64_t my_tiles = n_tiles > blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t n_groups = (my_tiles + NSLOT - 1) / NSLOT;

  if (threadIdx.x == 0) {
    for (int s = 0; s < n_ring; ++s) {
      mbar_init(&w_full[s], 1);
      mbar_init(&w_empty[s], 1);
    }
    for (int t = 0; t < 2; ++t) {
      mbar_init(&in_ready[t], EPI_WARPS);
      mbar_init(&acc_full[t], 1);
      mbar_init(&st_done[t], 1);
      for (int s = 0; s < 4; ++s) {
        mbar_init(&a_full[4 * t + s], EPI_WARPS);
        mbar_init(&a_empty[4 * t + s], 1);
      }
    }
    for (int q = 0; q < 4; ++q) {
      mbar_init(&dot_bar[q], NWG);
      mbar_init(&dot_free[q], 1);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < P.L * W; i += blockDim.x) bias_s[i] = P.bias[i];
  for (int i = threadIdx.x; i < W; i += blockDim.x) wout_s[i] = P.wout[i];
  if (P.first_staged)
    for (int i = threadIdx.x; i < P.n_first; i += blockDim.x) first_s[i] = P.first[i];
  // split mode: one tile in flight, its stages' accumulators alternate between two halves
  const uint32_t tmem_cols = (uint32_t)(SPLIT ? 2 * W : NSLOT * W);
  if (warp == 0) tmem_alloc(tmem_base, tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_base;

  if (warp == 4 * NWG) {
    // ---------------- TMA producer ----------------
    if (lane == 0 && !P.stall) {
      for (int s = 0; s < P.n_stages; ++s) {
        prefetch_map(&maps.m[P.st_map[s]]);
        if (SPLIT && P.st_kind[s] != kBwd) prefetch_map(&maps.m[P.st_map_lo[s]]);
      }
      uint32_t slot = 0, ep = 1;
      int64_t armed = 0;  // weight loads issued
      for (int64_t pr = 0; pr < n_groups; ++pr) {
        for (int s = 0; s < P.n_stages; ++s) {
          const int n_src = (SPLIT && P.st_kind[s] != kBwd) ? 2 : 1;  // W_hi (then W_lo) per chunk
          const int n_t = (kJoint0 && s == 0) ? 1 : NSLOT;  // a joint first stage reads each chunk once
          for (int t = 0; t < n_t; ++t) {
            for (int c = 0; c < P.st_panels[s]; ++c) {
              for (int kk = 0; kk < 64 / kKChunk; ++kk) {
                for (int h = 0; h < kNSplit; ++h) {
                  for (int src = 0; src < n_src; ++src) {
                    if (!mbar_wait(&w_empty[slot], ep, abort_flag, err, 201, lim)) goto producer_done;
                    mbar_arrive_expect_tx(&w_full[slot], chunk_bytes);
                    tma_load_2d(ring + slot * chunk_bytes, &maps.m[src ? P.st_map_lo[s] : P.st_map[s]],
                                &w_full[slot], 64 * c + kKChunk * kk, h * NW);
                    ++armed;
                    if (++slot == n_ring) {
                      slot = 0;
                      ep ^= 1;
                    }
                  }
                }
              }
            }
          }
        }
      }
    producer_done:
      // No load may still be writing shared memory when the CTA exits.  On the abort path
      // the MMA issuer stops waiting for the chunks, so wait here (bounded, whatever the abort
      // flag says) for the last n_ring loads, the only ones not yet consumed; load j went to
      // ring slot j mod n_ring with phase parity (j / n_ring) mod 2.
      for (int64_t j = armed > n_ring ? armed - n_ring : 0; j < armed; ++j)
        mbar_wait_drain(&w_full[j % n_ring], (uint32_t)((j / n_ring) & 1), lim);
    }
  } else if (warp == 4 * NWG + 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      // phase parities: ring, in_ready (one bit per slot), a_full (one bit per slot and buffer)
      uint32_t slot = 0, wf = 0, irp = 0u, ap = 0u;
      uint32_t sc = 0u;  // split mode: stages issued so far (the accumulator half is sc & 1)
      const uint32_t idesc = idesc_bf16(128, NW, false, false);
      bool issued = false;
      // VJP: the input panels of a slot (activations or deltas of its tile) are also the
      // scratch rows the weight-gradient GEMM reads; they are written out with TMA stores
      // issued here once the epilogue has published them.  Before the slot's next
      // acc_full (after which the epilogue overwrites the panels) the stores must have
      // read shared memory.
      auto store_panels = [&](int t, int map, int layer, int64_t tile) {
        for (int c = 0; c < W / 64; ++c)
          tma_store_2d(&maps.m[map], apan + (4 * t + c) * kPanelBytes, 64 * c,
                       (int)(layer * P.npts_pad + tile * kTile));
        bulk_commit_group();
      };
      for (int64_t pr = 0; pr < n_groups; ++pr) {
        const int64_t tile0 = blockIdx.x + (NSLOT * pr) * (int64_t)gridDim.x;
        for (int s = 0; s < P.n_stages; ++s) {
          const bool fsplit = SPLIT && P.st_kind[s] != kBwd;
          // split mode, stages after the first: the epilogue publishes each input panel as soon
          // as it has drained the previous stage's matching accumulator columns, and this stage
          // accumulates into the other TMEM half, so its MMAs overlap the rest of that drain
          const bool per_panel = SPLIT && s > 0;
          if (kJoint0 && s == 0) {
            // joint first stage: both tiles' feature panels, each weight chunk applied to both
            for (int t = 0; t < 2; ++t) {
              if (!mbar_wait(&in_ready[t], (irp >> t) & 1u, abort_flag, err, 301, lim)) goto mma_done;
              irp ^= 1u << t;
            }
            tc_fence_after();
            const int np = P.st_panels[0];
            for (int c = 0; c < np; ++c) {
              const int as = c & 3;
              if (c >= 1) {  // panels after the first are published one by one (both tiles)
                for (int t = 0; t < 2; ++t) {
                  const int bit = 4 * t + as;
                  if (!mbar_wait(&a_full[bit], (ap >> bit) & 1u, abort_flag, err, 302, lim)) goto mma_done;
                  ap ^= 1u << bit;
                }
                tc_fence_after();
              }
              const uint32_t a0 = smem_u32(apan + as * kPanelBytes), a1 = smem_u32(apan + (4 + as) * kPanelBytes);
              for (int kk = 0; kk < 64 / kKChunk; ++kk) {
                for (int h = 0; h < kNSplit; ++h) {
                  if (!mbar_wait(&w_full[slot], wf, abort_flag, err, 303, lim)) goto mma_done;
                  tc_fence_after();
                  const uint32_t bbase = smem_u32(ring + slot * chunk_bytes);
#pragma unroll
                  for (int j = 0; j < kKChunk / 16; ++j) {
                    const int ks = kk * (kKChunk / 16) + j;
                    const uint64_t bd = desc_sw(bbase + 32 * j, 16, 16 * kKChunk, 2 * kKChunk);
                    const uint32_t accum = (c > 0 || ks > 0) ? 1u : 0u;
                    mma_bf16(tmem + h * NW, desc_sw128(a0 + 32 * ks, 16, 1024), bd, idesc, accum);
                    mma_bf16(tmem + W + h * NW, desc_sw128(a1 + 32 * ks, 16, 1024), bd, idesc, accum);
                  }
                  issued = true;
                  mma_commit(&w_empty[slot]);
                  if (++slot == n_ring) {
                    slot = 0;
                    wf ^= 1;
                  }
                }
              }
              if (c + 4 < np) {  // both buffers take panel c + 4 next
                mma_commit(&a_empty[as]);
                mma_commit(&a_empty[4 + as]);
              }
            }
            mma_commit(&acc_full[0]);
            mma_commit(&acc_full[1]);
            continue;
          }
          // the first stage's panel 0 comes with in_ready, its later panels one by one (a_full)
          const bool stream = per_panel || s == 0;
          for (int t = 0; t < NSLOT; ++t) {
            const bool store_in = MODE == 1 && P.st_in_arr[s] >= 0 && tile0 + t * gridDim.x < n_tiles;
            if (!per_panel) {
              if (!mbar_wait(&in_ready[t], (irp >> t) & 1u, abort_flag, err, 301, lim)) goto mma_done;
              irp ^= 1u << t;
              tc_fence_after();
              if (store_in && !stream)
                store_panels(t, P.st_in_arr[s] ? P.map_dlt : P.map_act, P.st_in_layer[s],
                             tile0 + t * gridDim.x);
            }
            const uint32_t dbase = tmem + (SPLIT ? (sc & 1u) * (uint32_t)W : (uint32_t)(t * W));
            const int np = P.st_panels[s];
            for (int c = 0; c < np; ++c) {
              const int as = c & 3;
              if (per_panel || (s == 0 && c >= 1)) {  // published one by one (in_ready brought panel 0)
                const int bit = 4 * t + as;
                if (!mbar_wait(&a_full[4 * t + as], (ap >> bit) & 1u, abort_flag, err, 302, lim)) goto mma_done;
                ap ^= 1u << bit;
                tc_fence_after();
              }
              if (stream && store_in)  // this panel goes out to the scratch as soon as it is in
                tma_store_2d(&maps.m[P.st_in_arr[s] ? P.map_dlt : P.map_act], apan + (4 * t + c) * kPanelBytes,
                             64 * c, (int)(P.st_in_layer[s] * P.npts_pad + (tile0 + t * gridDim.x) * kTile));
              const uint32_t abase = smem_u32(apan + (4 * t + as) * kPanelBytes);
              const uint32_t lbase = smem_u32(apan + (4 + as) * kPanelBytes);  // low parts (SPLIT)
              for (int kk = 0; kk < 64 / kKChunk; ++kk) {
                for (int h = 0; h < kNSplit; ++h) {
                  const uint32_t dcol = dbase + h * NW;
                  // W_hi chunk: A_hi (and, split, A_lo) against it
                  if (!mbar_wait(&w_full[slot], wf, abort_flag, err, 303, lim)) goto mma_done;
                  tc_fence_after();
                  {
                    const uint32_t bbase = smem_u32(ring + slot * chunk_bytes);
#pragma unroll
                    for (int j = 0; j < kKChunk / 16; ++j) {
                      const int ks = kk * (kKChunk / 16) + j;  // K=16 step within the 64-wide panel
                      const uint64_t bd = desc_sw(bbase + 32 * j, 16, 16 * kKChunk, 2 * kKChunk);
                      mma_bf16(dcol, desc_sw128(abase + 32 * ks, 16, 1024), bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                      if (fsplit) mma_bf16(dcol, desc_sw128(lbase + 32 * ks, 16, 1024), bd, idesc, 1u);
                    }
                  }
                  issued = true;
                  mma_commit(&w_empty[slot]);
                  if (++slot == n_ring) {
                    slot = 0;
                    wf ^= 1;
                  }
                  if (fsplit) {
                    // W_lo chunk: A_hi against it
                    if (!mbar_wait(&w_full[slot], wf, abort_flag, err, 303, lim)) goto mma_done;
                    tc_fence_after();
                    const uint32_t bbase = smem_u32(ring + slot * chunk_bytes);
#pragma unroll
                    for (int j = 0; j < kKChunk / 16; ++j) {
                      const int ks = kk * (kKChunk / 16) + j;
                      mma_bf16(dcol, desc_sw128(abase + 32 * ks, 16, 1024),
                               desc_sw(bbase + 32 * j, 16, 16 * kKChunk, 2 * kKChunk), idesc, 1u);
                    }
                    mma_commit(&w_empty[slot]);
                    if (++slot == n_ring) {
                      slot = 0;
                      wf ^= 1;
                    }
                  }
                }
              }
              if (c + 4 < np) mma_commit(&a_empty[4 * t + as]);  // the buffer takes panel c + 4 next
            }
            if (stream && store_in) bulk_commit_group();
            if (MODE == 1) bulk_wait_read_all();
            mma_commit(&acc_full[t]);
          }
          if (SPLIT) ++sc;
        }
        if (MODE == 1) {
          // the deltas of the last stage: stored, then the feature pass of the next group may
          // overwrite the panels
          for (int t = 0; t < NSLOT; ++t) {
            if (!mbar_wait(&in_ready[t], (irp >> t) & 1u, abort_flag, err, 304, lim)) goto mma_done;
            irp ^= 1u << t;
            if (tile0 + t * gridDim.x < n_tiles) store_panels(t, P.map_dlt, P.tail_layer, tile0 + t * gridDim.x);
            bulk_wait_read_all();
            mbar_arrive(&st_done[t]);
          }
        }
      }
    mma_done:
      if (MODE == 1) bulk_wait_all();
      if (issued) {
        // drain: every issued MMA completes before TMEM is released (matters on the
        // abort path; otherwise the epilogue has already waited for all of them)
        mma_commit(drain_bar);
        mbar_wait_drain(drain_bar, 0, lim);
      }
    }
  } else {
    // ---------------- epilogue warps 0 .. 4*NWG-1 ----------------
    const int q = warp & 3, g = warp >> 2;
    const int r = q * 32 + lane;                 // row of the tile = TMEM lane
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    uint32_t ae = 0u, af = 0u, sdp = 0u, dot_uses = 0u;  // phase parities (a_empty per slot and buffer; per slot)
    uint32_t sc = 0u;  // split mode: stages drained so far (the accumulator half is sc & 1), as the MMA issuer counts
    // offset of this thread's CW sigma' values of (layer, tile, 64-column chunk c) in P.Sg
    auto sg_off = [&](int layer, int64_t tile, int c) -> int64_t {
      return ((((int64_t)layer * n_tiles + tile) * (W / 64) + c) * NWG + g) * (kTile * CW) + (int64_t)r * CW;
    };
    const float bout = P.theta[P.offbout];
    const float inv_N = 1.f / (float)P.N;
    float v[CW];
    // split VJP (ReLU): the masks 1[u_l > 0] of this thread's 16 columns of every 64-column
    // chunk, per hidden layer, as bits (local memory), in place of a scratch round trip
    uint16_t mk[SPLIT ? 4 * kMaxLayers : 1];
    double bsum = 0.0;  // VJP: this row's share of sum scale * v_i (warps of column group 0)
    double fsum = 0.0;  // VJP: this row's share of sum scale * v_i * f(x_i) (the virtual loss)
    for (int64_t pr = 0; pr < n_groups; ++pr) {
      // per-slot point data, kept in scalars (slot t selects with a conditional)
      const int64_t tile0 = blockIdx.x + (NSLOT * pr) * (int64_t)gridDim.x;
      const int64_t tile1 = tile0 + gridDim.x;  // two slots only; may be past the end: a dummy tile
      float x0[3], x1[3] = {0.f, 0.f, 0.f}, sv0, sv1 = 0.f;
      int m0[3] = {0, 0, 0}, m1[3] = {0, 0, 0};  // coordinate numerators (exact FFN phases, VJP)
      bool valid0, valid1 = false;
      {
        auto setup = [&](int64_t tile, float* x, int* m, float& sv, bool& valid) {
          const int64_t pt = tile * kTile + r;
          valid = pt < P.npts;
          int64_t gi = valid ? (P.idx ? (int64_t)P.idx[pt] : pt) : 0;
          const bool in_range = gi >= 0 && gi < P.n_grid;
          if (!in_range) gi = 0;
          point_coords(gi, P.N, P.d, x);
          if (MODE == 1 && KIND == INRCT_FFN_RELU) point_numerators(gi, P.N, P.d, m);
          const bool weighted = valid && in_range && (!P.fov || in_fov(gi, P.N));
          sv = (MODE == 1 && weighted) ? P.scale * P.v[gi] : 0.f;
        };
        setup(tile0, x0, m0, sv0, valid0);
        if (NSLOT == 2) setup(tile1, x1, m1, sv1, valid1);
      }
      if (MODE == 1 && g == 0) bsum += (double)sv0 + (double)sv1;
      // ---- first stage input ----
      for (int t = 0; t < NSLOT; ++t) {
        const int64_t prow_t = (t ? tile1 : tile0) * kTile + r;  // scratch row (padded to the tile)
        const bool store_t = (t ? tile1 : tile0) < n_tiles;      // dummy tiles write nowhere
        const int64_t tile_t = t ? tile1 : tile0;
        const float xt[3] = {t ? x1[0] : x0[0], t ? x1[1] : x0[1], t ? x1[2] : x0[2]};
        const int mt[3] = {t ? m1[0] : m0[0], t ? m1[1] : m0[1], t ? m1[2] : m0[2]};
        if (MODE == 1 && pr > 0) {
          // the previous group's last deltas are still being stored from these panels
          if (!warp_wait(&st_done[t], (sdp >> t) & 1u, abort_flag, err, 405, lim)) goto epi_done;
          sdp ^= 1u << t;
        }
        if constexpr (kJoint0) {
          // Joint first stage (grid evaluation of a Fourier-feature network): each pass writes
          // feature panel c of both tiles, the features' coefficients read once for the two
          // points of this thread.  Waits and arrivals as in the loop below, for both slots.
          // (Reading the coefficients once per two points and publishing every panel as soon as
          // it is written took the 501^3 evaluation from 128.5 to 119.7 ms.)
          if (t == 1) continue;  // slot 1's panels were written with slot 0's
          for (int c = 0; c < P.in_panels; ++c) {
            const int as = c & 3, f0 = 32 * c + 8 * g;
            float v0[16], v1[16];  // [0, 8) cos, [8, 16) sin of tile 0's and tile 1's point
            auto feature = [&](int i, const float4 bf) {
              float p0 = fmaf(bf.y, x0[1], bf.x * x0[0]);
              float p1 = fmaf(bf.y, x1[1], bf.x * x1[0]);
              if (P.d == 3) {
                p0 = fmaf(bf.z, x0[2], p0);
                p1 = fmaf(bf.z, x1[2], p1);
              }
              four_feat_fast(p0, &v0[8 + i], &v0[i]);
              four_feat_fast(p1, &v1[8 + i], &v1[i]);
            };
            // the table's source is uniform for the launch: one branch, not a select per read
            if (FC.n) {
#pragma unroll
              for (int i = 0; i < 8; ++i) feature(i, FC.c[f0 + i]);
            } else if (P.first_staged) {
#pragma unroll
              for (int i = 0; i < 8; ++i) feature(i, first_s[f0 + i]);
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i) feature(i, __ldg(P.first + f0 + i));
            }
            if (c >= 4) {  // streamed panels: the MMAs must have read panel c - 4 of both tiles
#pragma unroll
              for (int tt = 0; tt < 2; ++tt) {
                const int bit = 4 * tt + as;
                if (!warp_wait(&a_empty[bit], (ae >> bit) & 1u, abort_flag, err, 401, lim)) goto epi_done;
                ae ^= 1u << bit;
              }
            }
            st_panel_row<8>(apan + as * kPanelBytes, r, g, v0);
            st_panel_row<8>(apan + as * kPanelBytes, r, 4 + g, v0 + 8);
            st_panel_row<8>(apan + (4 + as) * kPanelBytes, r, g, v1);
            st_panel_row<8>(apan + (4 + as) * kPanelBytes, r, 4 + g, v1 + 8);
            {  // every panel is published: panel 0 with in_ready, the others with a_full
              fence_async_smem();
              if (c == 0) tc_fence_before();  // both slots' accumulators were drained before
              __syncwarp();
              if (lane == 0) {
                if (c == 0) {
                  mbar_arrive(&in_ready[0]);
                  mbar_arrive(&in_ready[1]);
                } else {
                  mbar_arrive(&a_full[as]);
                  mbar_arrive(&a_full[4 + as]);
                }
              }
            }
          }
        } else {
        for (int c = 0; c < P.in_panels; ++c) {
          const int col0 = 64 * c + CW * g;
          if (KIND == INRCT_FFN_RELU) {
            // features f0 .. f0+7 of this thread: cos into panel columns 8g.., sin into 32+8g..
            static_assert(NWG == 4, "the interleaved feature panels assume 4 column groups");
            const int f0 = 32 * c + 8 * g;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float4 bf = P.first_staged ? first_s[f0 + i] : __ldg(P.first + f0 + i);
              if (MODE == 1) {
                // the VJP decides ReLU masks downstream: the phase to an FP32 ulp of t
                feat_sincos(ffn_phase_exact(bf.x, bf.y, bf.z, mt, P.d, P.N, inv_N), &v[8 + i], &v[i]);
              } else {
                float ph = fmaf(bf.y, xt[1], bf.x * xt[0]);
                if (P.d == 3) ph = fmaf(bf.z, xt[2], ph);
                four_feat_fast(ph, &v[8 + i], &v[i]);  // v[0..7] cos, v[8..15] sin
              }
            }
            if (MODE == 1 && store_t) {
              store_row_bf16<8>(P.E + prow_t * (2 * P.F) + 64 * c + 8 * g, v);
              store_row_bf16<8>(P.E + prow_t * (2 * P.F) + 64 * c + 32 + 8 * g, v + 8);
            }
          } else {
            float cs[CW];
#pragma unroll
            for (int i = 0; i < CW; ++i) {
              const float4 w1 = P.first_staged ? first_s[col0 + i] : __ldg(P.first + col0 + i);
              const float z = fmaf(w1.x, xt[0], fmaf(w1.y, xt[1], fmaf(w1.z, xt[2], w1.w)));
              if (MODE == 1)
                __sincosf(z, &v[i], &cs[i]);
              else
                v[i] = __sinf(z);
            }
            if (MODE == 1 && store_t) {
              store_row_bf16<CW>(P.Sg + sg_off(0, tile_t, c), cs);
              if (c == 0 && g == 0) {
#pragma unroll
                for (int k = 0; k < 3; ++k)
                  P.Y16c[(int64_t)k * P.npts_pad + prow_t] = __float2bfloat16_rn(k < P.d ? xt[k] : 0.f);
              }
            }
          }
          const int as = c & 3;
          if (c >= 4) {  // streamed panel: the MMA must have read panel c - 4 from this buffer
            const int bit = 4 * t + as;
            if (!warp_wait(&a_empty[4 * t + as], (ae >> bit) & 1u, abort_flag, err, 401, lim)) goto epi_done;
            ae ^= 1u << bit;
          }
          if (KIND == INRCT_FFN_RELU) {
            st_panel_row<8>(apan + (4 * t + as) * kPanelBytes, r, g, v);
            st_panel_row<8>(apan + (4 * t + as) * kPanelBytes, r, 4 + g, v + 8);
            if (SPLIT) {
              st_panel_row_lo<8>(apan + (4 + as) * kPanelBytes, r, g, v);
              st_panel_row_lo<8>(apan + (4 + as) * kPanelBytes, r, 4 + g, v + 8);
            }
          } else {
            st_panel_row<CW>(apan + (4 * t + as) * kPanelBytes, r, (CW / 8) * g, v);
            if (SPLIT) st_panel_row_lo<CW>(apan + (4 + as) * kPanelBytes, r, (CW / 8) * g, v);
          }
          if (c == 0) {
            // panel 0 written and (program order) this slot's accumulator drained: the MMAs may
            // start; the later panels follow one by one
            fence_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&in_ready[t]);
          } else {
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_full[4 * t + as]);
          }
        }
        }
      }
      // ---- GEMM stages, alternating slots ----
      for (int s = 0; s < P.n_stages; ++s) {
        const int kind = P.st_kind[s], l = P.st_layer[s];
        const bool write_panel = s + 1 < P.n_stages;  // the next stage's input
        const bool write_lo = SPLIT && kind == kFwdHidden;  // the next stage is a split forward stage
        for (int t = 0; t < NSLOT; ++t) {
          const int64_t prow_t = (t ? tile1 : tile0) * kTile + r;
          const bool store_t = (t ? tile1 : tile0) < n_tiles;
          const bool valid_t = t ? valid1 : valid0;
          const float sv_t = t ? sv1 : sv0;
          const int64_t tile_t = t ? tile1 : tile0;
          const bool bwd = MODE == 1 && kind == kBwd;
          const bool pub = write_panel || MODE == 1;  // VJP: the last deltas are stored from the panels
          // split mode: each panel of the next stage's input is published as soon as it is written
          const bool per_panel_out = SPLIT && s + 1 < P.n_stages;
          const uint32_t hcol = SPLIT ? (sc & 1u) * (uint32_t)W : (uint32_t)(t * W);
          // backward: sigma'(u_{l-1}) of this tile; chunk c + 1 is fetched while chunk c is
          // processed, chunk 0 before the wait for the accumulator (a dummy tile reads nothing)
          uint4 sgn[CW / 8];
          if (bwd && !SPLIT) {
#pragma unroll
            for (int k = 0; k < CW / 8; ++k)
              sgn[k] = store_t ? reinterpret_cast<const uint4*>(P.Sg + sg_off(l - 1, tile_t, 0))[k]
                               : make_uint4(0, 0, 0, 0);
          }
          if (!warp_wait(&acc_full[t], (af >> t) & 1u, abort_flag, err, 402, lim)) goto epi_done;
          af ^= 1u << t;
          tc_fence_after();
          float dot = 0.f;
          // evaluation: the accumulator columns of two chunks are loaded behind one wait (W / 64
          // is 2 or 4); the VJP, which holds more live values, loads one chunk at a time
          constexpr int kPair = MODE == 0 ? 2 : 1;
          static_assert(kPair == 1 || CW == 16, "paired accumulator loads take 16 columns per chunk");
          for (int c2 = 0; c2 < W / 64; c2 += kPair) {
            float vv[kPair * CW];
            if constexpr (kPair == 2)
              tmem_ld16x2(tmem + lane_off + hcol + 64 * c2 + CW * g,
                          tmem + lane_off + hcol + 64 * (c2 + 1) + CW * g, vv);
            else
              tmem_ld<CW>(tmem + lane_off + hcol + 64 * c2 + CW * g, vv);
#pragma unroll
            for (int cc = 0; cc < kPair; ++cc) {
              const int c = c2 + cc;
              const int col0 = 64 * c + CW * g;
              float* v = vv + cc * CW;
              if (bwd && SPLIT) {
                // ReLU: delta_{l-1} = v * 1[u_{l-1} > 0], the mask bits this thread kept
                const uint32_t bits = mk[(l - 1) * 4 + c];
#pragma unroll
                for (int i = 0; i < CW; ++i) v[i] = ((bits >> i) & 1u) ? v[i] : 0.f;
              } else if (bwd) {
                // v = (W'_l^T delta_l) for layer l; delta_{l-1} = v * sigma'(u_{l-1})
                float sg[CW];
#pragma unroll
                for (int k = 0; k < CW / 8; ++k) {
                  const uint32_t u[4] = {sgn[k].x, sgn[k].y, sgn[k].z, sgn[k].w};
#pragma unroll
                  for (int e = 0; e < 4; ++e) {
                    sg[8 * k + 2 * e] = __uint_as_float(u[e] << 16);
                    sg[8 * k + 2 * e + 1] = __uint_as_float(u[e] & 0xffff0000u);
                  }
                }
                if (c + 1 < W / 64) {
#pragma unroll
                  for (int k = 0; k < CW / 8; ++k)
                    sgn[k] = store_t ? reinterpret_cast<const uint4*>(P.Sg + sg_off(l - 1, tile_t, c + 1))[k]
                                     : make_uint4(0, 0, 0, 0);
                }
                if (KIND == INRCT_FFN_RELU) {
#pragma unroll
                  for (int i = 0; i < CW; ++i) v[i] = sg[i] > 0.f ? v[i] : 0.f;
                } else {
#pragma unroll
                  for (int i = 0; i < CW; ++i) v[i] *= sg[i];
                }
              } else {
                const float4* bl = reinterpret_cast<const float4*>(bias_s + (size_t)l * W + col0);
                float cs[CW];
#pragma unroll
                for (int i4 = 0; i4 < CW / 4; ++i4) {
                  const float4 bb = bl[i4];
                  const float bq[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
                  for (int k = 0; k < 4; ++k) {
                    const int i = 4 * i4 + k;
                    const float z = v[i] + bq[k];
                    if (KIND == INRCT_FFN_RELU) {
                      v[i] = fmaxf(z, 0.f);
                      if (MODE == 1) cs[i] = z > 0.f ? 1.f : 0.f;
                    } else if (MODE == 1) {
                      __sincosf(z, &v[i], &cs[i]);
                    } else {
                      v[i] = __sinf(z);
                    }
                  }
                }
                if (SPLIT && kind == kFwdHidden) {
                  // the masks stay with this thread: it drains the same row and columns of the
                  // backward stage of layer l + 1
                  uint32_t bits = 0u;
#pragma unroll
                  for (int i = 0; i < CW; ++i) bits |= (cs[i] > 0.f ? 1u : 0u) << i;
                  mk[l * 4 + c] = (uint16_t)bits;
                }
                if (MODE == 1 && store_t) {
                  if (kind == kFwdLast)  // a_{L-1} is not a panel (the panels take delta_{L-1})
                    store_row_bf16<CW>(P.Act + ((int64_t)l * P.npts_pad + prow_t) * W + col0, v);
                  else if (!SPLIT)       // sigma'(u_l); a_l itself goes out from the panels
                    store_row_bf16<CW>(P.Sg + sg_off(l, tile_t, c), cs);
                }
                if (kind == kFwdLast) {
                  // f(x) = w_out . a_{L-1} + b_out: this thread's share of the dot product
                  const float4* wo = reinterpret_cast<const float4*>(wout_s + col0);
#pragma unroll
                  for (int i4 = 0; i4 < CW / 4; ++i4) {
                    const float4 ww = wo[i4];
                    dot = fmaf(v[4 * i4], ww.x, dot);
                    dot = fmaf(v[4 * i4 + 1], ww.y, dot);
                    dot = fmaf(v[4 * i4 + 2], ww.z, dot);
                    dot = fmaf(v[4 * i4 + 3], ww.w, dot);
                  }
                  if (MODE == 1) {
                    // delta_{L-1} = scale v_i * w_out * sigma'(u_{L-1})
#pragma unroll
                    for (int i4 = 0; i4 < CW / 4; ++i4) {
                      const float4 ww = wo[i4];
                      v[4 * i4] = sv_t * ww.x * cs[4 * i4];
                      v[4 * i4 + 1] = sv_t * ww.y * cs[4 * i4 + 1];
                      v[4 * i4 + 2] = sv_t * ww.z * cs[4 * i4 + 2];
                      v[4 * i4 + 3] = sv_t * ww.w * cs[4 * i4 + 3];
                    }
                    if (store_t && c == 0 && g == 0) P.Y16o[prow_t] = __float2bfloat16_rn(sv_t);
                  }
                }
              }
              if (pub) {
                st_panel_row<CW>(apan + (4 * t + c) * kPanelBytes, r, (CW / 8) * g, v);
                if (write_lo) st_panel_row_lo<CW>(apan + (4 + c) * kPanelBytes, r, (CW / 8) * g, v);
              }
              if (per_panel_out) {
                // this warp's rows and columns of panel c are written (and its accumulator
                // columns read): with the other 15 warps' arrivals the MMAs may take the panel
                fence_async_smem();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&a_full[4 * t + c]);
              }
            }
          }
          if (!per_panel_out) {
            if (pub) fence_async_smem();
            tc_fence_before();
            __syncwarp();
            if (pub && lane == 0) mbar_arrive(&in_ready[t]);
          }
          if (kind == kFwdLast) {
            // f = b_out + sum of the NWG column-group partial dot products of row r; one
            // scratch buffer per row quarter, released by its summing warp (dot_free)
            if (dot_uses > 0) {
              if (!warp_wait(&dot_free[q], (dot_uses - 1) & 1u, abort_flag, err, 406, lim)) goto epi_done;
            }
            dotp[g * kTile + r] = dot;
            __syncwarp();
            if (lane == 0) mbar_arrive(&dot_bar[q]);
            if (g == 0) {
              if (!warp_wait(&dot_bar[q], dot_uses & 1u, abort_flag, err, 404, lim)) goto epi_done;
              float f = bout;
#pragma unroll
              for (int q2 = 0; q2 < NWG; ++q2) f += dotp[q2 * kTile + r];
              __syncwarp();
              if (lane == 0) mbar_arrive(&dot_free[q]);
              if (MODE == 0) {
                if (valid_t) P.out[prow_t] = f;
              } else {
                fsum += (double)sv_t * (double)f;  // sv_t is 0 for points without weight
              }
            }
            ++dot_uses;
          }
        }
        if (SPLIT) ++sc;
      }
    }
    if (MODE == 1 && g == 0) {
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        bsum += __shfl_down_sync(0xffffffffu, bsum, o);
        fsum += __shfl_down_sync(0xffffffffu, fsum, o);
      }
      if (lane == 0) {
        P.bias_part[(int64_t)blockIdx.x * 4 + q] = bsum;
        P.vloss_part[(int64_t)blockIdx.x * 4 + q] = fsum;
      }
    }
  epi_done:;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, tmem_cols);
  }
}

// Launches the tile kernel instance for (mode, kind) with the needed shared memory.
int launch_tile(int mode, const Net& n, const Maps& maps, const TileProg& P, int grid, int* err,
                cudaStream_t st);

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

constexpr int kTileNWG = 4;  // epilogue warpgroups of the tile kernel

size_t tile_smem_base(int mode) {
  return 8 * (size_t)kPanelBytes + (size_t)ring_bytes(mode) + 8 * (size_t)kTileBars +
         sizeof(float) * (size_t)kTileNWG * kTile;
}
// Biases and output weights staged, and the first-layer table too when it fits
bool first_fits(const Net& n) {
  const size_t n_first = n.kind == INRCT_SIREN ? n.W : n.F;
  return tile_smem_base(1) + sizeof(float) * ((size_t)n.L * n.W + n.W) + 16 * n_first <= 232448;
}
size_t tile_smem(const Net& n, int mode = 0) {
  const size_t n_first = n.kind == INRCT_SIREN ? n.W : n.F;
  return tile_smem_base(mode) + sizeof(float) * ((size_t)n.L * n.W + n.W) + (first_fits(n) ? 16 * n_first : 0);
}


template <int MODE, int KIND, bool SPLIT>
int launch_tile_t(const Net& n, const Maps& maps, const TileProg& P, int grid, int* err, cudaStream_t st) {
  const size_t sm = tile_smem(n, MODE);
  cudaError_t e = cudaFuncSetAttribute(mlp_tile_kernel<MODE, KIND, kTileNWG, SPLIT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) {
    set_error("tile kernel shared memory (%zu bytes): %s", sm, cudaGetErrorString(e));
    return INRCT_ERR_CUDA;
  }
  typename FirstArg<MODE, KIND, SPLIT>::type fc{};
  if constexpr (std::is_same_v<typename FirstArg<MODE, KIND, SPLIT>::type, FirstConst>) {
    if (n.B_host && n.F <= kMaxConstFirst) {  // the same entries prep_all_kernel writes
      fc.n = n.F;
      for (int f = 0; f < n.F; ++f) {
        const float* b = n.B_host + (size_t)f * n.d;
        fc.c[f] = make_float4(b[0], b[1], n.d == 3 ? b[2] : 0.f, 0.f);
      }
    }
  }
  mlp_tile_kernel<MODE, KIND, kTileNWG, SPLIT><<<grid, 32 * (4 * kTileNWG + 2), sm, st>>>(maps, P, fc, err);
  INRCT_CHECK_LAUNCH("mlp tile kernel");
  return INRCT_OK;
}

// Instances: evaluation (two slots) for both kinds; VJP with two slots for SIREN and with
// split forward operands (one slot) for ReLU networks.
int launch_tile(int mode, const Net& n, const Maps& maps, const TileProg& P, int grid, int* err,
                cudaStream_t st) {
  if (mode == 0)
    return n.kind == INRCT_SIREN ? launch_tile_t<0, INRCT_SIREN, false>(n, maps, P, grid, err, st)
                                 : launch_tile_t<0, INRCT_FFN_RELU, false>(n, maps, P, grid, err, st);
  return n.kind == INRCT_SIREN ? launch_tile_t<1, INRCT_SIREN, false>(n, maps, P, grid, err, st)
                               : launch_tile_t<1, INRCT_FFN_RELU, true>(n, maps, P, grid, err, st);
}
constexpr size_t kGemmSmem = (size_t)kGemmStages * kGemmStageBytes + 2048 + 1024;

struct TcWeights {
  __nv_bfloat16* Wb[kMaxLayers];
  __nv_bfloat16* WbT[kMaxLayers];
  __nv_bfloat16* Wlo[kMaxLayers];  // low parts of Wb for the split forward stages (ReLU networks)
  float* bias;
  float4* first;  // SIREN: W entries; FFN: F entries
  float* wout;    // W
};

// Layers handled by the MMA stages: FFN 0..L-1, SIREN 1..L-1 (the SIREN first layer is FP32).
int first_mma_layer(const Net& n) { return n.kind == INRCT_SIREN ? 1 : 0; }

// The VJP of a ReLU network runs its forward stages on split operands (see mlp_tile_kernel).
bool split_vjp(const Net& n, int mode) { return mode == 1 && n.kind == INRCT_FFN_RELU; }

// BF16 weights (and their transposes) plus FP32 biases, laid out in order.
void weights_layout(const Net& n, Carver& c, TcWeights* w) {
  w->bias = c.take<float>((size_t)n.L * n.W);
  w->first = c.take<float4>((size_t)(n.kind == INRCT_SIREN ? n.W : n.F));
  w->wout = c.take<float>((size_t)n.W);
  for (int l = 0; l < kMaxLayers; ++l) w->Wb[l] = w->WbT[l] = w->Wlo[l] = nullptr;
  for (int l = first_mma_layer(n); l < n.L; ++l) {
    w->Wb[l] = c.take<__nv_bfloat16>((size_t)n.in_dim[l] * n.out_dim[l]);
    w->WbT[l] = c.take<__nv_bfloat16>((size_t)n.in_dim[l] * n.out_dim[l]);
    if (n.kind == INRCT_FFN_RELU) w->Wlo[l] = c.take<__nv_bfloat16>((size_t)n.in_dim[l] * n.out_dim[l]);
  }
}

size_t weights_bytes(const Net& n) {
  Carver c(nullptr, 0);
  TcWeights w;
  weights_layout(n, c, &w);
  return c.off + 256;
}

// One launch converts every MMA layer of theta (omega0 folded for SIREN).
int prep_weights(const Net& n, const float* theta, const TcWeights& w, cudaStream_t st) {
  PrepTable T;
  memset(&T, 0, sizeof(T));
  int64_t most = 0;
  for (int l = first_mma_layer(n); l < n.L; ++l) {
    const int i = T.n++;
    T.out[i] = n.out_dim[l];
    T.in[i] = n.in_dim[l];
    T.offW[i] = n.offW[l];
    T.offb[i] = n.offb[l];
    T.Wb[i] = w.Wb[l];
    T.WbT[i] = w.WbT[l];
    T.Wlo[i] = w.Wlo[l];
    T.bias[i] = w.bias + (int64_t)l * n.W;
    most = std::max<int64_t>(most, (int64_t)n.in_dim[l] * n.out_dim[l]);
  }
  T.permF = n.kind == INRCT_FFN_RELU ? n.F : 0;
  T.kind = n.kind;
  T.d = n.d;
  T.W = n.W;
  T.n_first = n.kind == INRCT_SIREN ? n.W : n.F;
  T.offW0 = n.offW[0];
  T.offb0 = n.offb[0];
  T.offWout = n.offW[n.L];
  T.B = n.B;
  T.first = w.first;
  T.wout = w.wout;
  const float sc = n.kind == INRCT_SIREN ? n.omega0 : 1.f;
  most = std::max<int64_t>(most, T.n_first);
  dim3 grd((unsigned)std::min<int64_t>(ceil_div(most, 256), 512), T.n + 1);
  prep_all_kernel<<<grd, 256, 0, st>>>(theta, T, sc);
  INRCT_CHECK_LAUNCH("weight preparation");
  return INRCT_OK;
}

int set_smem_attr(const void* fn, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) {
    set_error("shared memory attribute: %s", cudaGetErrorString(e));
    return INRCT_ERR_CUDA;
  }
  return INRCT_OK;
}

// Builds the stage program and its weight maps.
int build_prog(const Net& n, const TcWeights& w, int mode, TileProg* P, Maps* maps) {
  memset(P, 0, sizeof(*P));
  P->mode = mode;
  P->kind = n.kind;
  P->d = n.d;
  P->F = n.F;
  P->W = n.W;
  P->L = n.L;
  P->omega0 = n.omega0;
  P->B = n.B;
  P->bias = w.bias;
  P->first = w.first;
  P->n_first = n.kind == INRCT_SIREN ? n.W : n.F;
  P->first_staged = first_fits(n) ? 1 : 0;
  P->wout = w.wout;
  P->offW0 = n.offW[0];
  P->offb0 = n.offb[0];
  P->offWout = n.offW[n.L];
  P->offbout = n.offb[n.L];
  P->in_panels = n.kind == INRCT_FFN_RELU ? n.K0 / 64 : n.W / 64;
  int s = 0, mi = 0;
  for (int l = first_mma_layer(n); l < n.L; ++l, ++s) {
    P->st_kind[s] = l == n.L - 1 ? kFwdLast : kFwdHidden;
    P->st_layer[s] = l;
    // input of a forward stage: a_{l-1}; for the first MMA layer of an FFN, the features (E)
    P->st_in_arr[s] = l == 0 ? -1 : 0;
    P->st_in_layer[s] = l - 1;
    P->st_panels[s] = n.in_dim[l] / 64;
    INRCT_REQUIRE(s == 0 || P->st_panels[s] <= 4, "tile kernel: stage %d has %d input panels", s,
                  P->st_panels[s]);
    P->st_map[s] = mi;
    // a ring slot holds out_dim / kNSplit output rows x 64 K (see mlp_tile_kernel)
    INRCT_TRY(make_map(&maps->m[mi++], w.Wb[l], n.in_dim[l], n.out_dim[l], kKChunk, n.out_dim[l] / kNSplit,
                       2 * kKChunk));
    P->st_map_lo[s] = -1;
    if (split_vjp(n, mode)) {
      INRCT_REQUIRE(w.Wlo[l] != nullptr, "tile kernel: no low parts of layer %d", l);
      P->st_map_lo[s] = mi;
      INRCT_TRY(make_map(&maps->m[mi++], w.Wlo[l], n.in_dim[l], n.out_dim[l], kKChunk,
                         n.out_dim[l] / kNSplit, 2 * kKChunk));
    }
    INRCT_REQUIRE(n.out_dim[l] == n.W, "tile kernel: MMA layer %d has %d outputs, expected %d", l,
                  n.out_dim[l], n.W);
  }
  if (mode == 1) {
    for (int l = n.L - 1; l >= 1; --l, ++s) {
      P->st_kind[s] = kBwd;
      P->st_layer[s] = l;
      P->st_in_arr[s] = 1;  // delta_l
      P->st_in_layer[s] = l;
      P->st_panels[s] = n.out_dim[l] / 64;
      P->st_map[s] = mi;
      P->st_map_lo[s] = -1;
      // W'_l^T is [in][out]: rows = in (the MMA N), K = out; chunks of in / kNSplit rows
      INRCT_REQUIRE(n.in_dim[l] == n.W, "tile kernel: backward stage %d has N=%d, expected %d", l,
                    n.in_dim[l], n.W);
      INRCT_TRY(make_map(&maps->m[mi++], w.WbT[l], n.out_dim[l], n.in_dim[l], kKChunk, n.in_dim[l] / kNSplit,
                         2 * kKChunk));
    }
  }
  P->n_stages = s;
  // after the last stage the panels hold delta_{l-1} of its layer (a backward stage) or
  // delta_{L-1} (a network whose only MMA layer is the last one)
  P->tail_layer = P->st_kind[s - 1] == kBwd ? P->st_layer[s - 1] - 1 : P->st_layer[s - 1];
  P->map_act = mi;  // filled by the caller, which owns the scratch
  P->map_dlt = mi + 1;
  INRCT_REQUIRE(mi + 2 <= kMaxJobs, "tile kernel: %d tensor maps", mi + 2);
  return INRCT_OK;
}

}  // namespace

bool tc_supported(const Net& n, char* why, size_t len) {
  if (n.kind == INRCT_HASH) {
    snprintf(why, len, "the hash-encoded INR has no tensor-core path");
    return false;
  }
  if (n.W != 128 && n.W != 256) {
    snprintf(why, len, "width %d unsupported (128 or 256)", n.W);
    return false;
  }
  if (n.kind == INRCT_SIREN && n.L < 2) {
    snprintf(why, len, "SIREN needs at least 2 hidden layers on the tensor-core path");
    return false;
  }
  if (n.kind == INRCT_FFN_RELU && (n.F % 32) != 0) {
    snprintf(why, len, "n_feat=%d must be a multiple of 32", n.F);
    return false;
  }
  if (n.kind == INRCT_FFN_RELU && 2 * n.F > 2048) {
    snprintf(why, len, "n_feat=%d too large (<= 1024)", n.F);
    return false;
  }
  if (std::max(tile_smem(n, 0), tile_smem(n, 1)) > 232448) {  // all of it is dynamic
    snprintf(why, len, "network too large for the tile kernel's shared memory (%zu bytes)", tile_smem(n));
    return false;
  }
  return true;
}

size_t tc_weights_bytes(const Net& n) { return weights_bytes(n); }

int tc_prepare(const Net& n, const float* theta, void* buf, size_t bytes, cudaStream_t st) {
  Carver c(buf, bytes);
  TcWeights w;
  weights_layout(n, c, &w);
  if (!buf || !c.ok) {
    set_error("tensor-core weights: buffer of %zu bytes too small (need %zu)", bytes, weights_bytes(n));
    return INRCT_ERR_WORKSPACE;
  }
  return prep_weights(n, theta, w, st);
}

size_t tc_eval_ws_bytes(const Net& n) { return weights_bytes(n) + 256; }

int tc_eval(const Net& n, const float* theta, int N, int64_t npts, float* image, void* ws, size_t ws_bytes,
            cudaStream_t st, const void* prepared) {
  Carver c(ws, ws_bytes);
  TcWeights w;
  weights_layout(n, c, &w);
  if (!ws || !c.ok) {
    set_error("inr_eval_grid (bf16): workspace of %zu bytes too small (need %zu)", ws_bytes,
              tc_eval_ws_bytes(n));
    return INRCT_ERR_WORKSPACE;
  }
  if (prepared) {
    Carver pc(const_cast<void*>(prepared), SIZE_MAX);
    weights_layout(n, pc, &w);
  } else {
    INRCT_TRY(prep_weights(n, theta, w, st));
  }
  int* err = nullptr;
  INRCT_TRY(status_word(st, &err));
  Maps maps;  // per call: the kernel takes a copy at launch
  TileProg P;
  INRCT_TRY(build_prog(n, w, 0, &P, &maps));
  P.wait_ns = g_wait_ns.load();
  P.stall = g_stall_loads.load();
  P.theta = theta;
  P.N = N;
  P.n_grid = npts;
  P.fov = 0;  // evaluation: the caller masks the image
  P.npts = npts;
  P.out = image;
  const int64_t tiles = (npts + kTile - 1) / kTile;
  const int grid = (int)std::min<int64_t>((tiles + 1) / 2, num_sms());  // tiles go in pairs per CTA
  prof_mark(kMarkEvalKernel, st);
  INRCT_TRY(launch_tile(0, n, maps, P, grid, err, st));
  prof_mark(kMarkEvalDone, st);
  return INRCT_OK;
}

namespace {

struct TcVjpWs {
  TcWeights w;
  __nv_bfloat16 *E, *Act, *Dlt, *Sg, *Y16c, *Y16o;
  float* part;
  double* bias_part;
  double* vloss_part;
  int64_t pad;
  size_t part_floats;
};

// Split-K GEMM plan.  The split count fills about one wave of CTAs (one CTA per SM);
// for_sizing: the largest plan any device could use (workspace sizing).
GemmPlan plan_gemm(const Net& n, int64_t K, int64_t* part_floats, bool for_sizing = false) {
  GemmPlan G;
  memset(&G, 0, sizeof(G));
  G.K = K;
  const int64_t nch = (K + 63) / 64;
  int mt = 0;  // m-tiles over all jobs (see the job list below)
  for (int l = 0; l < n.L; ++l)
    mt += (l == 0 && n.kind == INRCT_SIREN) ? n.W / 128 : (n.W / 128) * ((n.in_dim[l] + 255) / 256);
  mt += n.W / 128;
  const int per_wave = for_sizing ? kMaxSplits : std::max(1, num_sms() / std::max(mt, 1));
  int S = (int)std::min<int64_t>(nch, std::min(kMaxSplits, per_wave));
  const int64_t per_ch = (nch + S - 1) / S;
  S = (int)((nch + per_ch - 1) / per_ch);
  G.S = S;
  G.per_split = per_ch * 64;
  int j = 0;
  int64_t off = 0;
  const double mult = n.kind == INRCT_SIREN ? n.omega0 : 1.0;
  auto add = [&](GemmJob J) {
    J.mtiles = J.M / 128;
    J.part_off = off;
    off += (int64_t)S * J.M * (J.N + 32);
    G.job[j++] = J;
  };
  // map indices: 0 = X of layer l at 3l, Y at 3l + 1, Y16 at 3l + 2 (filled in by the caller)
  for (int l = 0; l < n.L; ++l) {
    const int in = n.in_dim[l];
    if (l == 0 && n.kind == INRCT_SIREN) {
      GemmJob J{};
      J.M = n.W;
      J.N = 0;
      J.has_ones = 1;
      J.has_y16 = 1;
      J.mx = 3 * l;
      J.my16 = 3 * l + 2;
      J.offW = n.offW[0];
      J.ldW = n.d;
      J.w_src = 1;
      J.w_cols = n.d;
      J.offb = n.offb[0];
      J.mult = mult;
      add(J);
      continue;
    }
    for (int n0 = 0; n0 < in; n0 += 256) {
      GemmJob J{};
      J.M = n.W;
      J.N = std::min(256, in - n0);
      J.n0 = n0;
      J.has_ones = n0 == 0;
      J.mx = 3 * l;
      J.my = 3 * l + 1;
      J.offW = n.offW[l];
      J.ldW = in;
      J.w_src = 0;
      J.w_cols = J.N;
      J.offb = n0 == 0 ? n.offb[l] : -1;
      J.mult = mult;
      J.permF = (l == 0 && n.kind == INRCT_FFN_RELU) ? n.F : 0;
      add(J);
    }
  }
  {  // output layer: dw_out = sum_points (scale v_i) a_{L-1}
    GemmJob J{};
    J.M = n.W;
    J.N = 0;
    J.has_y16 = 1;
    J.mx = 3 * n.L;
    J.my16 = 3 * n.L + 2;
    J.offW = n.offW[n.L];
    J.ldW = 1;  // dw_out[m] is column 0 of row m
    J.w_src = 1;
    J.w_cols = 1;
    J.offb = -1;
    J.mult = 1.0;
    add(J);
  }
  G.n_jobs = j;
  int cta = 0;
  for (int q = 0; q < j; ++q) {
    G.cta_begin[q] = cta;
    cta += G.job[q].mtiles * S;
  }
  G.cta_begin[j] = cta;
  *part_floats = off;
  return G;
}

size_t vjp_layout(const Net& n, int64_t chunk, void* ws, size_t cap, TcVjpWs* out, bool* ok) {
  Carver c(ws, cap);
  TcVjpWs w;
  weights_layout(n, c, &w.w);
  const int64_t pad = (chunk + kTile - 1) / kTile * kTile;
  w.pad = pad;
  w.E = n.kind == INRCT_FFN_RELU ? c.take<__nv_bfloat16>((size_t)pad * n.K0) : nullptr;
  w.Act = c.take<__nv_bfloat16>((size_t)pad * n.L * n.W);
  w.Dlt = c.take<__nv_bfloat16>((size_t)pad * n.L * n.W);
  // sigma'(u_l) of the SIREN (cos u_l); the split VJP of ReLU networks keeps its masks as bits
  w.Sg = n.kind == INRCT_SIREN ? c.take<__nv_bfloat16>((size_t)pad * std::max(n.L - 1, 1) * n.W) : nullptr;
  w.Y16c = c.take<__nv_bfloat16>((size_t)16 * pad);
  w.Y16o = c.take<__nv_bfloat16>((size_t)16 * pad);
  int64_t pf;
  plan_gemm(n, chunk, &pf, true);
  w.part_floats = (size_t)pf;
  w.part = c.take<float>((size_t)pf);
  w.bias_part = c.take<double>(4 * 1024);   // 4 per tile-kernel CTA
  w.vloss_part = c.take<double>(4 * 1024);  // 4 per tile-kernel CTA
  if (out) *out = w;
  if (ok) *ok = c.ok;
  return c.off + 256;
}

}  // namespace

size_t tc_vjp_ws_bytes(const Net& n, int64_t n_idx) {
  const int64_t chunk = n_idx < kVjpChunk ? n_idx : kVjpChunk;
  return vjp_layout(n, chunk, nullptr, 0, nullptr, nullptr);
}

int tc_vjp(const Net& n, const float* theta, int N, const int32_t* idx, int64_t n_idx, const float* v,
           double scale, double* grad_f64, float* grad_f32, double* value_out, void* ws, size_t ws_bytes,
           cudaStream_t st, const void* prepared) {
  const int64_t chunk = n_idx < kVjpChunk ? n_idx : kVjpChunk;
  TcVjpWs w;
  bool ok;
  const size_t need = vjp_layout(n, chunk, ws, ws_bytes, &w, &ok);
  if (!ws || !ok) {
    set_error("inr_weighted_vjp (bf16): workspace of %zu bytes too small (need %zu)", ws_bytes, need);
    return INRCT_ERR_WORKSPACE;
  }
  int* err = nullptr;
  INRCT_TRY(status_word(st, &err));
  if (prepared) {  // weights converted once by the caller (grad_step)
    Carver pc(const_cast<void*>(prepared), SIZE_MAX);
    weights_layout(n, pc, &w.w);
  } else {
    INRCT_TRY(prep_weights(n, theta, w.w, st));
  }
  Maps tmaps, gmaps;  // per call: each launch takes a copy
  TileProg P;
  INRCT_TRY(build_prog(n, w.w, 1, &P, &tmaps));
  P.wait_ns = g_wait_ns.load();
  P.stall = g_stall_loads.load();
  P.theta = theta;
  P.N = N;
  int64_t ng = 1;
  for (int k = 0; k < n.d; ++k) ng *= N;
  P.n_grid = ng;
  P.fov = n.fov;
  P.v = v;
  P.scale = (float)scale;
  P.E = w.E;
  P.Act = w.Act;
  P.Dlt = w.Dlt;
  P.Sg = w.Sg;
  // panel stores: the scratch as [L * pad rows][W], 128-row x 64-column boxes like the panels
  INRCT_TRY(make_map(&tmaps.m[P.map_act], w.Act, n.W, (uint64_t)n.L * w.pad, 64, kTile));
  INRCT_TRY(make_map(&tmaps.m[P.map_dlt], w.Dlt, n.W, (uint64_t)n.L * w.pad, 64, kTile));
  P.Y16c = w.Y16c;
  P.Y16o = w.Y16o;
  P.bias_part = w.bias_part;
  P.vloss_part = w.vloss_part;
  P.npts_pad = w.pad;
  const bool split = split_vjp(n, 1);  // one tile in flight per CTA, else two
  INRCT_TRY(set_smem_attr((const void*)tn_gemm_kernel, kGemmSmem));
  for (int64_t c0 = 0; c0 < n_idx; c0 += chunk) {
    const int64_t np = std::min(chunk, n_idx - c0);
    P.idx = idx + c0;
    P.npts = np;
    const int64_t tiles = (np + kTile - 1) / kTile;
    if (c0 == 0) prof_mark(kMarkVjpKernel, st);
    const int64_t per_cta = split ? tiles : (tiles + 1) / 2;
    const int tile_grid = (int)std::max<int64_t>(1, std::min<int64_t>(per_cta, num_sms()));
    INRCT_REQUIRE(tile_grid <= 1024, "tile grid %d exceeds the bias partial buffer", tile_grid);
    INRCT_TRY(launch_tile(1, n, tmaps, P, tile_grid, err, st));
    if (c0 == 0) prof_mark(kMarkVjpKernelDone, st);
    // split-K weight-gradient GEMMs over this chunk's points
    int64_t pf;
    GemmPlan G = plan_gemm(n, np, &pf);
    for (int l = 0; l < n.L; ++l) {
      INRCT_TRY(make_map(&gmaps.m[3 * l], w.Dlt + (int64_t)l * w.pad * n.W, n.W, np, 64, 64));
      if (l == 0 && n.kind == INRCT_SIREN) {
        INRCT_TRY(make_map(&gmaps.m[3 * l + 2], w.Y16c, w.pad, 16, 64, 16));
      } else if (l == 0) {
        INRCT_TRY(make_map(&gmaps.m[3 * l + 1], w.E, n.K0, np, 64, 64));
      } else {
        INRCT_TRY(make_map(&gmaps.m[3 * l + 1], w.Act + (int64_t)(l - 1) * w.pad * n.W, n.W, np, 64, 64));
      }
    }
    INRCT_TRY(make_map(&gmaps.m[3 * n.L], w.Act + (int64_t)(n.L - 1) * w.pad * n.W, n.W, np, 64, 64));
    INRCT_TRY(make_map(&gmaps.m[3 * n.L + 2], w.Y16o, w.pad, 16, 64, 16));
    G.wait_ns = P.wait_ns;
    tn_gemm_kernel<<<G.cta_begin[G.n_jobs], 192, kGemmSmem, st>>>(gmaps, G, w.part, err);
    INRCT_CHECK_LAUNCH("tn gemm");
    int maxe = 0;
    for (int q = 0; q < G.n_jobs; ++q)
      maxe = std::max(maxe, G.job[q].M * (G.job[q].w_cols + 1));
    G.bpart = w.bias_part;
    G.vpart = w.vloss_part;
    G.value_out = value_out;
    G.n_bpart = 4 * tile_grid;
    G.off_bout = n.offb[n.L];
    gemm_reduce_kernel<<<dim3(ceil_div(maxe, 256), G.n_jobs + 1), 256, 0, st>>>(G, w.part, c0 > 0, grad_f64);
    INRCT_CHECK_LAUNCH("gemm reduce");
  }
  if (grad_f32) INRCT_TRY(f64_to_f32(grad_f64, grad_f32, n.p, st));
  return INRCT_OK;
}


namespace {
__global__ void gemm_diag_reduce_kernel(const float* __restrict__ part, int S, int M, int ldc,
                                        float* __restrict__ C) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * ldc) return;
  double s = 0.0;
  for (int q = 0; q < S; ++q) s += (double)part[(int64_t)q * M * ldc + e];
  C[e] = (float)s;
}

GemmPlan diag_plan(int64_t K, int M, int N, bool y16, int64_t* pf) {
  GemmPlan G;
  memset(&G, 0, sizeof(G));
  G.K = K;
  const int64_t nch = (K + 63) / 64;
  int S = (int)std::min<int64_t>(nch, kMaxSplits);
  const int64_t per_ch = (nch + S - 1) / S;
  S = (int)((nch + per_ch - 1) / per_ch);
  G.S = S;
  G.per_split = per_ch * 64;
  GemmJob J{};
  J.M = M;
  J.N = N;
  J.has_ones = 1;
  J.has_y16 = y16 ? 1 : 0;
  J.mx = 0;
  J.my = 1;
  J.my16 = 2;
  J.mtiles = M / 128;
  G.job[0] = J;
  G.n_jobs = 1;
  G.cta_begin[0] = 0;
  G.cta_begin[1] = J.mtiles * S;
  *pf = (int64_t)S * M * (N + 32);
  return G;
}
}  // namespace

size_t gemm_tn_ws_bytes(int64_t K, int M, int N) {
  int64_t pf;
  diag_plan(K, M, N, true, &pf);
  return align_up(sizeof(float) * pf, 256) + 256;
}

__global__ void sincospi_diag_kernel(const float* __restrict__ x, float* __restrict__ s, float* __restrict__ c,
                                     int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) feat_sincos(0.5f * x[i], s + i, c + i);  // the feature code path, phase x / 2
}

int sincospi_diag(const float* x, float* s, float* c, int64_t n, cudaStream_t st) {
  INRCT_REQUIRE(x && s && c && n > 0, "sincospi: NULL buffer or n <= 0");
  sincospi_diag_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(x, s, c, n);
  INRCT_CHECK_LAUNCH("sincospi (diagnostic)");
  return INRCT_OK;
}

int gemm_tn(const void* X, const void* Y, const void* Y16, int64_t K, int M, int N, float* C, void* ws,
            size_t ws_bytes, cudaStream_t st) {
  INRCT_REQUIRE(X && C && K > 0 && K < (int64_t)1 << 31, "gemm_tn: bad X, C or K");
  INRCT_REQUIRE(M > 0 && M % 128 == 0 && M <= 4096, "gemm_tn: M=%d must be a multiple of 128", M);
  INRCT_REQUIRE(N >= 0 && N <= 256 && N % 64 == 0 && (N == 0 || Y), "gemm_tn: N=%d must be 0..256, step 64",
                N);
  int64_t pf;
  GemmPlan G = diag_plan(K, M, N, Y16 != nullptr, &pf);
  Carver c(ws, ws_bytes);
  float* part = c.take<float>((size_t)pf);
  if (!ws || !c.ok) {
    set_error("gemm_tn: workspace of %zu bytes too small (need %zu)", ws_bytes, gemm_tn_ws_bytes(K, M, N));
    return INRCT_ERR_WORKSPACE;
  }
  Maps maps;
  INRCT_TRY(make_map(&maps.m[0], X, M, K, 64, 64));
  if (N > 0) INRCT_TRY(make_map(&maps.m[1], Y, N, K, 64, 64));
  if (Y16) INRCT_TRY(make_map(&maps.m[2], Y16, K, 16, 64, 16));
  int* err = nullptr;
  INRCT_TRY(status_word(st, &err));
  G.wait_ns = g_wait_ns.load();
  INRCT_TRY(set_smem_attr((const void*)tn_gemm_kernel, kGemmSmem));
  tn_gemm_kernel<<<G.cta_begin[1], 192, kGemmSmem, st>>>(maps, G, part, err);
  INRCT_CHECK_LAUNCH("tn gemm (diagnostic)");
  const int ldc = N + 32;
  gemm_diag_reduce_kernel<<<ceil_div((int64_t)M * ldc, 256), 256, 0, st>>>(part, G.S, M, ldc, C);
  INRCT_CHECK_LAUNCH("tn gemm reduce (diagnostic)");
  return INRCT_OK;
}

int tc_device_status(cudaStream_t st, int* code) {
  int* word = nullptr;
  INRCT_TRY(status_word(st, &word));
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, word, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(word, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error("device status: %s", cudaGetErrorString(e));
    return INRCT_ERR_CUDA;
  }
  *code = h;
  return INRCT_OK;
}

int tc_status_resolve(cudaStream_t st) {
  int* word = nullptr;
  return status_word(st, &word);
}

void tc_set_wait_limit(unsigned long long ns) { g_wait_ns.store(ns ? ns : kWaitTimeoutNs); }
void tc_set_stall_loads(int on) { g_stall_loads.store(on ? 1 : 0); }

}  // namespace inrct
