// FP32 SIMT path of the INR: the plain comparator of the BF16 tensor-core path.
//
// Computes E{f_theta} on the grid (Sec. 3) and the weighted Jacobian-transpose
// product sum_i w_i grad_theta f(x_i) with w_i = scale * v_i at listed points
// (Sec. 3, Eq. 2; with every grid point listed it is the full gradient).
//
// Layout: theta follows inrct.h (W row-major [out][in], then b).  The forward
// reads a transposed FP32 copy W^T [in][out] so that the thread computing
// output o reads consecutive addresses; the backward chain reads W itself for
// the same reason.  A VJP runs per chunk of at most kVjpChunk points:
//   1. forward at the chunk, storing the layer-1 input E and the
//      pre-activations Z_l (scratch grows with the chunk, never with the grid);
//   2. backward chain delta_l = (W_{l+1}^T delta_{l+1}) * sigma'(z_l), stored;
//   3. dW_l = sum_points delta_l a_{l-1}^T and db_l = sum delta_l as a split-K
//      SIMT GEMM with FP32 partials per split (64x64 tiles; the scalar output layer
//      by a one-thread-per-column kernel);
//   4. reduction of the partials into the FP64 gradient: FP32 within a warp, FP64
//      across warps in a fixed order (accumulated over chunks).
//
// Hash-encoded INR (Sec. 4, "Hash Enc."): the layer-1 input is gathered from the
// tables at theta[0, n_table) by the forward kernel; the backward kernel finishes
// with g = W_1^T delta_1 per point and scatters w_v g into the 2^d vertex entries
// of every level with FP64 atomics (the encoding is linear in the entries).
#include <math.h>

#include "mlp.cuh"

namespace inrct {

namespace {

struct NetDev {
  int kind, d, F, W, L, K0, N;
  float omega0;
  const float* B;
  int hL, hF, hlog2T;
  unsigned hdense;  // bit l: level l is looked up densely
  float rcp2N;      // 1 / (2N) rounded to FP32
  int fov;          // listed points outside the field of view carry no weight
  int hres[kMaxHashLevels];
};

struct LayerOffs {
  int64_t W[kMaxLayers], b[kMaxLayers], Wt[kMaxLayers];
};

NetDev dev_of(const Net& n, int N) {
  NetDev d;
  d.kind = n.kind;
  d.d = n.d;
  d.F = n.F;
  d.W = n.W;
  d.L = n.L;
  d.K0 = n.K0;
  d.N = N;
  d.omega0 = n.omega0;
  d.B = n.B;
  d.hL = n.hL;
  d.hF = n.hF;
  d.hlog2T = n.hlog2T;
  d.hdense = 0;
  d.rcp2N = 1.0f / (2.0f * (float)N);
  d.fov = n.fov;
  for (int l = 0; l < kMaxHashLevels; ++l) {
    d.hres[l] = l < n.hL ? n.hres[l] : 0;
    if (l < n.hL) {
      int64_t cells = 1;
      for (int a = 0; a < n.d; ++a) cells *= (int64_t)n.hres[l] + 1;
      if (cells <= ((int64_t)1 << n.hlog2T)) d.hdense |= 1u << l;
    }
  }
  return d;
}

// Offsets of the transposed copies of layers 0..L-1 inside the W^T buffer.
int64_t wt_layout(const Net& n, LayerOffs* lo) {
  int64_t off = 0;
  for (int l = 0; l <= n.L; ++l) {
    lo->W[l] = n.offW[l];
    lo->b[l] = n.offb[l];
    lo->Wt[l] = off;
    if (l < n.L) off += (int64_t)n.in_dim[l] * n.out_dim[l];
  }
  return off;
}

__device__ __forceinline__ int64_t grid_size(const NetDev& n) {
  return n.d == 3 ? (int64_t)n.N * n.N * n.N : (int64_t)n.N * n.N;
}

__device__ __forceinline__ float act(const NetDev& n, float z) {
  return n.kind != INRCT_SIREN ? fmaxf(z, 0.f) : sinf(n.omega0 * z);
}
__device__ __forceinline__ float dact(const NetDev& n, float z) {
  return n.kind != INRCT_SIREN ? (z > 0.f ? 1.f : 0.f) : n.omega0 * cosf(n.omega0 * z);
}

// Level l of the hash encoding at the grid point with per-axis indices k[0..D): the
// table entries of its 2^D surrounding vertices and their multilinear weights.  The
// level coordinate (2k + 1) N_l / (2N) is split exactly into its integer part c0 and
// remainder r: while the numerator stays below 2^24 (exact in FP32) the quotient from
// the FP32 reciprocal is within one of the floor, and one integer correction makes it
// exact; larger numerators divide in 32 or 64-bit integers.  The fraction is r / (2N)
// in FP32 (exact when 2N is a power of two).  D is a template parameter so that every
// loop unrolls and the vertex state stays in registers.
template <int D>
__device__ __forceinline__ void hash_vertices(const NetDev& n, int l, const int* k, uint32_t (&ent)[1 << D],
                                              float (&w)[1 << D]) {
  const uint32_t Nl = (uint32_t)n.hres[l];
  const uint32_t twoN = 2u * (uint32_t)n.N;
  uint32_t c0[D];
  float fr[D];
  // (2k + 1) N_l < 2N N_l
  const uint64_t bound = (uint64_t)twoN * Nl;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    uint32_t rem;
    if (bound <= (1u << 24)) {
      // |num * fl(1/2N) - num / 2N| < 2 num 2^-24 / 2N < 1: truncation is off by at most one
      const uint32_t num = (2u * (uint32_t)k[a] + 1u) * Nl;
      uint32_t q = (uint32_t)((float)num * n.rcp2N);
      int r = (int)num - (int)(q * twoN);
      if (r < 0) {
        q -= 1;
        r += (int)twoN;
      } else if (r >= (int)twoN) {
        q += 1;
        r -= (int)twoN;
      }
      c0[a] = q;
      rem = (uint32_t)r;
    } else if (bound <= 0xFFFFFFFFull) {
      const uint32_t num = (2u * (uint32_t)k[a] + 1u) * Nl;
      c0[a] = num / twoN;
      rem = num - c0[a] * twoN;
    } else {
      const uint64_t num = (2ull * (uint32_t)k[a] + 1ull) * Nl;
      c0[a] = (uint32_t)(num / twoN);
      rem = (uint32_t)(num - (uint64_t)c0[a] * twoN);
    }
    fr[a] = (float)rem * n.rcp2N;
  }
  const bool dense = (n.hdense >> l) & 1u;
  const uint32_t mask = (1u << n.hlog2T) - 1u;
  constexpr uint32_t kPrime[3] = {1u, 2654435761u, 805459861u};
#pragma unroll
  for (int v = 0; v < (1 << D); ++v) {
    float wv = 1.f;
    uint32_t lin = 0, stride = 1, h = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const uint32_t bit = (v >> a) & 1;
      const uint32_t c = c0[a] + bit;
      wv *= bit ? fr[a] : 1.f - fr[a];
      lin += c * stride;  // dense levels have (N_l + 1)^D <= T <= 2^24 entries: no wrap
      stride *= Nl + 1u;
      h ^= c * kPrime[a];  // 32-bit unsigned, wraps by definition
    }
    ent[v] = dense ? lin : (h & mask);
    w[v] = wv;
  }
}

// Features of level l at the point: sum_v w_v table[ent_v][f], f < F.
template <int D>
__device__ __forceinline__ void hash_gather(const NetDev& n, const float* __restrict__ theta, int l,
                                            const int* k, float* out) {
  uint32_t ent[1 << D];
  float w[1 << D];
  hash_vertices<D>(n, l, k, ent, w);
  const float* tab = theta + ((int64_t)l << n.hlog2T) * n.hF;
  if (n.hF == 2) {
    // both features of a vertex in one 8-byte load (theta is 256-byte aligned and every
    // table and entry offset is even)
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int v = 0; v < (1 << D); ++v) {
      const float2 e = __ldg(reinterpret_cast<const float2*>(tab) + ent[v]);
      a0 = fmaf(w[v], e.x, a0);
      a1 = fmaf(w[v], e.y, a1);
    }
    out[0] = a0;
    out[1] = a1;
    return;
  }
  for (int f = 0; f < n.hF; ++f) {
    float a = 0.f;
#pragma unroll
    for (int v = 0; v < (1 << D); ++v) a = fmaf(w[v], __ldg(tab + (int64_t)ent[v] * n.hF + f), a);
    out[f] = a;
  }
}

// Table gradient of level l at one point per lane: entry ent_v, feature f receives
// w_v g[f].  Called by all 32 lanes of a warp together (ok = false: the lane adds
// nothing).  Runs of consecutive lanes whose vertex is the same (level, entry) are summed
// by a segmented scan (5 shuffle steps, no divergence) and the last lane of each run
// issues the one atomic: neighbouring points of a sorted index set share vertices at
// coarse levels.  A key that recurs after another key simply starts a new run, so the
// result holds for any order of the points.
template <int D>
__device__ __forceinline__ void hash_scatter_warp(const NetDev& n, double* __restrict__ gtab, int l, const int* k,
                                                  const float* g, bool ok) {
  const unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  uint32_t ent[1 << D];
  float w[1 << D];
  if (ok) hash_vertices<D>(n, l, k, ent, w);
  double* gl = gtab + ((int64_t)(ok ? l : 0) << n.hlog2T) * n.hF;
#pragma unroll
  for (int v = 0; v < (1 << D); ++v) {
    const unsigned long long key = ok ? ((unsigned long long)l << 32) | ent[v] : ~0ull - lane;
    const unsigned long long kprev = __shfl_up_sync(kFull, key, 1);
    const bool head = lane == 0 || kprev != key;
    const bool next_head = __shfl_down_sync(kFull, (int)head, 1) != 0;  // lane 31: its own
    const bool tail = lane == 31 || next_head;
    // which of the five steps add the value of lane - 2^s (segmented scan: a lane stops
    // taking once the run's head has reached it)
    unsigned take = 0;
    bool f = head;
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const int off = 1 << st;
      const bool fu = __shfl_up_sync(kFull, (int)f, off) != 0;
      if (lane >= off && !f) {
        take |= 1u << st;
        f = fu;
      }
    }
    for (int ff = 0; ff < n.hF; ++ff) {
      float val = ok ? w[v] * g[ff] : 0.f;
#pragma unroll
      for (int st = 0; st < 5; ++st) {
        const float up = __shfl_up_sync(kFull, val, 1 << st);
        if (take & (1u << st)) val += up;
      }
      if (ok && tail) atomicAdd(gl + (int64_t)ent[v] * n.hF + ff, (double)val);
    }
  }
}

__global__ void transpose_w_kernel(const float* __restrict__ theta, int64_t offW, int out, int in,
                                   float* __restrict__ Wt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)out * in) return;
  const int k = (int)(t / out), o = (int)(t % out);
  Wt[t] = theta[offW + (int64_t)o * in + k];
}

constexpr int TP = 16;  // points per block

// Forward at npts points (grid order when idx == NULL).  Optional outputs:
// out_f[q] = f(x_q); E[q][K0] = layer-1 input; Z[l][q][W] = pre-activations.
__global__ void __launch_bounds__(256)
    simt_fwd_kernel(const __grid_constant__ NetDev net, const __grid_constant__ LayerOffs lo,
                    const float* __restrict__ theta,
                    const float* __restrict__ Wt, int64_t npts, const int32_t* __restrict__ idx,
                    float* __restrict__ out_f, float* __restrict__ E, float* __restrict__ Z) {
  extern __shared__ __align__(16) float sh[];
  __shared__ float xs[TP][3];
  __shared__ int ks[TP][3];
  __shared__ float red[TP][8];
  const int W = net.W, K0 = net.K0;
  const int Kmax = K0 > W ? K0 : W;
  float* bufA = sh;             // [TP][Kmax]
  float* bufB = sh + TP * Kmax;  // [TP][W]
  const int t = threadIdx.x;     // blockDim.x == W
  const int64_t p0 = (int64_t)blockIdx.x * TP;
  if (t < TP) {
    const int64_t q = p0 + t;
    int64_t i = q < npts ? (idx ? (int64_t)idx[q] : q) : 0;
    if (i < 0 || i >= grid_size(net)) i = 0;  // out-of-range indices contribute nothing
    float x[3];
    point_coords(i, net.N, net.d, x);
    xs[t][0] = x[0];
    xs[t][1] = x[1];
    xs[t][2] = x[2];
    ks[t][0] = (int)(i % net.N);
    ks[t][1] = (int)((i / net.N) % net.N);
    ks[t][2] = net.d == 3 ? (int)(i / ((int64_t)net.N * net.N)) : 0;
  }
  __syncthreads();
  if (net.kind == INRCT_HASH) {
    // one thread per (point, level): interpolate the level's features
    for (int e = t; e < TP * net.hL; e += W) {
      const int p = e / net.hL, l = e % net.hL;
      float* out = bufA + p * Kmax + l * net.hF;
      if (net.d == 3) hash_gather<3>(net, theta, l, ks[p], out);
      else hash_gather<2>(net, theta, l, ks[p], out);
    }
  } else if (net.kind == INRCT_FFN_RELU) {
    for (int e = t; e < TP * net.F; e += W) {
      const int p = e / net.F, f = e % net.F;
      const float* Bf = net.B + (int64_t)f * net.d;
      const int m[3] = {2 * ks[p][0] + 1 - net.N, 2 * ks[p][1] + 1 - net.N,
                        net.d == 3 ? 2 * ks[p][2] + 1 - net.N : 0};
      const float t = ffn_phase_exact(Bf[0], Bf[1], net.d == 3 ? Bf[2] : 0.f, m, net.d, net.N, 1.f / (float)net.N);
      float s, c;
      sincospif(2.f * t, &s, &c);
      bufA[p * Kmax + f] = c;
      bufA[p * Kmax + net.F + f] = s;
    }
  } else {
    for (int e = t; e < TP * net.d; e += W) bufA[(e / net.d) * Kmax + e % net.d] = xs[e / net.d][e % net.d];
  }
  __syncthreads();
  if (E) {
    for (int e = t; e < TP * K0; e += W) {
      const int p = e / K0, k = e % K0;
      if (p0 + p < npts) E[(p0 + p) * K0 + k] = bufA[p * Kmax + k];
    }
  }
  const float* in = bufA;
  int ld_in = Kmax, K = K0;
  for (int l = 0; l < net.L; ++l) {
    float acc[TP];
    const float bias = theta[lo.b[l] + t];
#pragma unroll
    for (int p = 0; p < TP; ++p) acc[p] = bias;
    const float* wt = Wt + lo.Wt[l];
    int k = 0;
    if ((ld_in & 3) == 0) {
      // four inputs per 16-byte shared load (a broadcast: every lane reads the same row)
      for (; k + 4 <= K; k += 4) {
        const float w0 = __ldg(wt + (int64_t)k * W + t), w1 = __ldg(wt + (int64_t)(k + 1) * W + t);
        const float w2 = __ldg(wt + (int64_t)(k + 2) * W + t), w3 = __ldg(wt + (int64_t)(k + 3) * W + t);
#pragma unroll
        for (int p = 0; p < TP; ++p) {
          const float4 x = *reinterpret_cast<const float4*>(in + p * ld_in + k);
          acc[p] = fmaf(x.x, w0, acc[p]);
          acc[p] = fmaf(x.y, w1, acc[p]);
          acc[p] = fmaf(x.z, w2, acc[p]);
          acc[p] = fmaf(x.w, w3, acc[p]);
        }
      }
    }
    for (; k < K; ++k) {
      const float w = __ldg(wt + (int64_t)k * W + t);
#pragma unroll
      for (int p = 0; p < TP; ++p) acc[p] = fmaf(in[p * ld_in + k], w, acc[p]);
    }
    float* out = (in == bufA) ? bufB : bufA;
    const int ld_out = (out == bufA) ? Kmax : W;
    __syncthreads();  // everyone done reading `in` (out may alias a previous input)
#pragma unroll
    for (int p = 0; p < TP; ++p) {
      if (Z && p0 + p < npts) Z[((int64_t)l * npts + p0 + p) * W + t] = acc[p];
      out[p * ld_out + t] = act(net, acc[p]);
    }
    __syncthreads();
    in = out;
    ld_in = ld_out;
    K = W;
  }
  if (out_f) {
    const float wo = theta[lo.W[net.L] + t];
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int p = 0; p < TP; ++p) {
      float v = in[p * ld_in + t] * wo;
#pragma unroll
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[p][warp] = v;
    }
    __syncthreads();
    if (t < TP && p0 + t < npts) {
      float s = theta[lo.b[net.L]];
      for (int w = 0; w < (W >> 5); ++w) s += red[t][w];
      out_f[p0 + t] = s;
    }
  }
}

// Backward chain at the chunk: delta_out = scale v_i, delta_{L-1} = delta_out w_out
// sigma'(z_{L-1}), delta_{l-1} = (W_l^T delta_l) sigma'(z_{l-1}).
// No launch bound: with one, ptxas caps this kernel's registers and spills (it needs
// about 72; any register count fits the largest block, 256 threads).
__global__ void simt_bwd_kernel(const __grid_constant__ NetDev net, const __grid_constant__ LayerOffs lo,
                    const float* __restrict__ theta, int64_t npts,
                    const int32_t* __restrict__ idx, const float* __restrict__ v, float scale,
                    const float* __restrict__ Z, float* __restrict__ Dl, float* __restrict__ dout,
                    double* __restrict__ gtab) {
  extern __shared__ __align__(16) float dsh[];  // [TP][W]
  __shared__ float dsc[TP];
  __shared__ int ksh[TP][3];  // per-axis grid indices (hash encoding)
  const int W = net.W, L = net.L;
  const int t = threadIdx.x;
  const int64_t p0 = (int64_t)blockIdx.x * TP;
  if (t < TP) {
    const int64_t q = p0 + t;
    float s = 0.f;
    if (q < npts) {
      const int64_t i = idx ? (int64_t)idx[q] : q;
      s = (i >= 0 && i < grid_size(net) && (!net.fov || in_fov(i, net.N))) ? scale * v[i] : 0.f;
      dout[q] = s;
      if (gtab && s != 0.f) {
        ksh[t][0] = (int)(i % net.N);
        ksh[t][1] = (int)((i / net.N) % net.N);
        ksh[t][2] = net.d == 3 ? (int)(i / ((int64_t)net.N * net.N)) : 0;
      }
    }
    dsc[t] = s;
  }
  __syncthreads();
  const float wo = theta[lo.W[L] + t];
#pragma unroll
  for (int p = 0; p < TP; ++p) {
    float d = 0.f;
    if (p0 + p < npts) {
      const float z = Z[((int64_t)(L - 1) * npts + p0 + p) * W + t];
      d = dsc[p] * wo * dact(net, z);
      Dl[((int64_t)(L - 1) * npts + p0 + p) * W + t] = d;
    }
    dsh[p * W + t] = d;
  }
  __syncthreads();
  for (int l = L - 1; l >= 1; --l) {
    float acc[TP];
#pragma unroll
    for (int p = 0; p < TP; ++p) acc[p] = 0.f;
    const float* Wl = theta + lo.W[l];  // [W][W], row o holds the weights of output o
    for (int o = 0; o < W; o += 4) {    // W is a multiple of 64
      const float w0 = __ldg(Wl + (int64_t)o * W + t), w1 = __ldg(Wl + (int64_t)(o + 1) * W + t);
      const float w2 = __ldg(Wl + (int64_t)(o + 2) * W + t), w3 = __ldg(Wl + (int64_t)(o + 3) * W + t);
#pragma unroll
      for (int p = 0; p < TP; ++p) {
        const float4 x = *reinterpret_cast<const float4*>(dsh + p * W + o);
        acc[p] = fmaf(x.x, w0, acc[p]);
        acc[p] = fmaf(x.y, w1, acc[p]);
        acc[p] = fmaf(x.z, w2, acc[p]);
        acc[p] = fmaf(x.w, w3, acc[p]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < TP; ++p) {
      float d = 0.f;
      if (p0 + p < npts) {
        const float z = Z[((int64_t)(l - 1) * npts + p0 + p) * W + t];
        d = acc[p] * dact(net, z);
        Dl[((int64_t)(l - 1) * npts + p0 + p) * W + t] = d;
      }
      dsh[p * W + t] = d;
    }
    __syncthreads();
  }
  if (gtab) {
    // hash tables: g = W_1^T delta_1 is the gradient of the layer-1 input (thread j < K0
    // computes column j for the block's points); each vertex entry of each level receives
    // its weight times the level's slice of g
    __shared__ float gsh[TP * kMaxHashInputs];
    const int K0 = net.K0;
    if (t < K0) {  // K0 <= 64 <= W
      const float* W0 = theta + lo.W[0];  // [W][K0]
      float acc[TP];
#pragma unroll
      for (int p = 0; p < TP; ++p) acc[p] = 0.f;
      for (int o = 0; o < W; o += 4) {
        const float w0 = __ldg(W0 + (int64_t)o * K0 + t), w1 = __ldg(W0 + (int64_t)(o + 1) * K0 + t);
        const float w2 = __ldg(W0 + (int64_t)(o + 2) * K0 + t), w3 = __ldg(W0 + (int64_t)(o + 3) * K0 + t);
#pragma unroll
        for (int p = 0; p < TP; ++p) {
          const float4 x = *reinterpret_cast<const float4*>(dsh + p * W + o);
          acc[p] = fmaf(x.x, w0, acc[p]);
          acc[p] = fmaf(x.y, w1, acc[p]);
          acc[p] = fmaf(x.z, w2, acc[p]);
          acc[p] = fmaf(x.w, w3, acc[p]);
        }
      }
#pragma unroll
      for (int p = 0; p < TP; ++p) gsh[p * K0 + t] = acc[p];
    }
    __syncthreads();
    // level-major items (a warp holds TP points of one level, two levels per warp); the
    // item count is rounded up to whole warps so that every lane of a warp takes part
    const int n_items = TP * net.hL;
    const int n_round = (n_items + 31) & ~31;
    for (int e = t; e < n_round; e += W) {  // W is a multiple of 32: warps stay whole
      const int l = e / TP, p = e % TP;
      const bool ok = e < n_items && p0 + p < npts && dsc[p] != 0.f;  // else ksh[p] is unset
      const float* g = gsh + p * K0 + (ok ? l : 0) * net.hF;
      if (net.d == 3) hash_scatter_warp<3>(net, gtab, l, ksh[p], g, ok);
      else hash_scatter_warp<2>(net, gtab, l, ksh[p], g, ok);
    }
  }
}

// C[o][k] (k <= K; column K is the bias) partial sums over one split of points:
//   C[o][k] = sum_q X[q][o] * Y'(q, k),  Y'(q, k) = f(Y[q][k]) for k < K, 1 for k = K,
// with f the identity (ymode 0), ReLU (1) or sin(omega0 .) (2).
constexpr int GT = 64, GK = 32;
constexpr int kDwLoads = GK * GT / 256;  // slab elements of X (and of Y) per thread

// One slab of GK points: X[q][o] and Y'(q, k) of this tile into registers (zero outside).
__device__ __forceinline__ void dw_load_slab(const float* __restrict__ X, int O, const float* __restrict__ Y,
                                             int K, int ymode, float omega0, int to, int tk, int64_t qb,
                                             int64_t q1, float (&xr)[kDwLoads], float (&yr)[kDwLoads]) {
#pragma unroll
  for (int r = 0; r < kDwLoads; ++r) {
    const int e = threadIdx.x + 256 * r;
    const int qq = e / GT, c = e % GT;
    const int64_t q = qb + qq;
    const int o = to * GT + c, k = tk * GT + c;
    float xv = 0.f, yv = 0.f;
    if (q < q1) {
      if (o < O) xv = __ldg(X + q * O + o);
      if (k < K) {
        yv = __ldg(Y + q * K + k);
        if (ymode == 1) yv = fmaxf(yv, 0.f);
        else if (ymode == 2) yv = sinf(omega0 * yv);
      }
    }
    xr[r] = xv;
    yr[r] = yv;
  }
}

// The slabs are double-buffered: while the FMAs of slab s read shared memory, the
// loads of slab s + 1 are in flight into registers; one barrier per slab.  The bias
// column (k = K) is a running sum of X kept by the blocks of k-tile 0, so K = 64 needs
// one k-tile, not two.
__global__ void __launch_bounds__(256)
    simt_dw_kernel(const float* __restrict__ X, int O, const float* __restrict__ Y, int K, int ymode,
                   float omega0, int64_t npts, int64_t per_split, float* __restrict__ part) {
  __shared__ __align__(16) float xs[2][GK][GT];
  __shared__ __align__(16) float ys[2][GK][GT];
  const int to = blockIdx.x, tk = blockIdx.y, sp = blockIdx.z;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t q0 = (int64_t)sp * per_split;
  const int64_t q1 = min(npts, q0 + per_split);
  float acc[4][4] = {};
  float accb[4] = {};
  float xr[kDwLoads], yr[kDwLoads];
  dw_load_slab(X, O, Y, K, ymode, omega0, to, tk, q0, q1, xr, yr);
  int buf = 0;
  for (int64_t qb = q0; qb < q1; qb += GK) {
#pragma unroll
    for (int r = 0; r < kDwLoads; ++r) {
      const int e = threadIdx.x + 256 * r;
      xs[buf][e / GT][e % GT] = xr[r];
      ys[buf][e / GT][e % GT] = yr[r];
    }
    __syncthreads();
    if (qb + GK < q1) dw_load_slab(X, O, Y, K, ymode, omega0, to, tk, qb + GK, q1, xr, yr);
#pragma unroll 8
    for (int qq = 0; qq < GK; ++qq) {
      const float4 a = *reinterpret_cast<const float4*>(&xs[buf][qq][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&ys[buf][qq][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      if (tk == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) accb[i] += av[i];
      }
    }
    buf ^= 1;  // the next slab goes to the other buffer: no barrier needed before its stores
  }
  const int ld = K + 1;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = to * GT + ty * 4 + i, k = tk * GT + tx * 4 + j;
      if (o < O && k < K) part[((int64_t)sp * O + o) * ld + k] = acc[i][j];
    }
  if (tk == 0 && tx == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int o = to * GT + ty * 4 + i;
      if (o < O) part[((int64_t)sp * O + o) * ld + K] = accb[i];
    }
  }
}

// dW of a one-row layer (the scalar output): part[s][0][k] = sum_q X[q] Y'(q, k) for
// k < K and part[s][0][K] = sum_q X[q].  Thread k streams the split's points: the Y
// rows are coalesced across threads, X[q] is one broadcast.
constexpr int kRowMinPoints = 32;
__global__ void __launch_bounds__(288)
    simt_dw_row_kernel(const float* __restrict__ X, const float* __restrict__ Y, int K, int ymode, float omega0,
                       int64_t npts, int64_t per_split, float* __restrict__ part) {
  const int k = threadIdx.x, sp = blockIdx.x;
  if (k > K) return;
  const int64_t q0 = (int64_t)sp * per_split;
  const int64_t q1 = min(npts, q0 + per_split);
  float acc0 = 0.f, acc1 = 0.f;
  int64_t q = q0;
  for (; q + 2 <= q1; q += 2) {
    float y0 = 1.f, y1 = 1.f;
    if (k < K) {
      y0 = __ldg(Y + q * K + k);
      y1 = __ldg(Y + (q + 1) * K + k);
      if (ymode == 1) {
        y0 = fmaxf(y0, 0.f);
        y1 = fmaxf(y1, 0.f);
      } else if (ymode == 2) {
        y0 = sinf(omega0 * y0);
        y1 = sinf(omega0 * y1);
      }
    }
    acc0 = fmaf(__ldg(X + q), y0, acc0);
    acc1 = fmaf(__ldg(X + q + 1), y1, acc1);
  }
  if (q < q1) {
    float y = 1.f;
    if (k < K) {
      y = __ldg(Y + q * K + k);
      if (ymode == 1) y = fmaxf(y, 0.f);
      else if (ymode == 2) y = sinf(omega0 * y);
    }
    acc0 = fmaf(__ldg(X + q), y, acc0);
  }
  part[(int64_t)sp * (K + 1) + k] = acc0 + acc1;
}

// grad[offW + o*K + k] (+)= sum_s part[s][o][k];  grad[offb + o] (+)= sum_s part[s][o][K].
// A block takes 32 consecutive entries; its 32 warps sum interleaved subsets of the
// splits (coalesced 128-byte rows, independent loads in flight) in FP32, then warp 0
// adds the 32 warp sums in FP64 in warp order, so the result does not depend on timing.
// (FP64 arithmetic is slow on this part: one FP64 add per partial would dominate.)
constexpr int kRedWarps = 32;
__global__ void __launch_bounds__(32 * kRedWarps)
    reduce_layer_kernel(const float* __restrict__ part, int S, int O, int K, int64_t offW, int64_t offb,
                        double mult, int accumulate, double* __restrict__ grad) {
  __shared__ double red[kRedWarps][32];
  const int ld = K + 1;
  const int64_t ent = (int64_t)O * ld;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  float s0 = 0.f, s1 = 0.f;
  if (e < ent) {
    int q = warp;
    for (; q + kRedWarps < S; q += 2 * kRedWarps) {
      s0 += part[(int64_t)q * ent + e];
      s1 += part[(int64_t)(q + kRedWarps) * ent + e];
    }
    if (q < S) s0 += part[(int64_t)q * ent + e];
  }
  red[warp][lane] = (double)s0 + (double)s1;
  __syncthreads();
  if (warp != 0 || e >= ent) return;
  double tot = 0.0;
#pragma unroll
  for (int w = 0; w < kRedWarps; ++w) tot += red[w][lane];
  tot *= mult;
  const int o = (int)(e / ld), k = (int)(e % ld);
  const int64_t dst = k < K ? offW + (int64_t)o * K + k : offb + o;
  grad[dst] = accumulate ? grad[dst] + tot : tot;
}

struct VjpWs {
  float* Wt;
  float* E;
  float* Z;
  float* D;
  float* dout;
  float* f;  // f(x) at the chunk's points (the virtual loss)
  float* part;
};

// *value (+)= sum_q w[q] f[q] in FP64: the virtual loss of Eq. 3 over one chunk, w the
// point weights scale * v_i of the backward kernel (zero for points without weight).  One
// block, fixed-order tree, so the result does not depend on scheduling.
__global__ void __launch_bounds__(256) weighted_sum_kernel(const float* __restrict__ w, const float* __restrict__ f,
                                                         int64_t n, int accumulate, double* __restrict__ value) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) s += (double)w[q] * (double)f[q];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *value = accumulate ? *value + sh[0] : sh[0];
}

// Point splits of one layer's dW: enough (tile, split) blocks for about four per SM of
// a 152-SM part, at least two slabs of points per split, at most kMaxDwSplits partials
// per entry.
// A fixed count (not the live SM count) keeps the workspace size a function of the
// network and the chunk alone.
constexpr int kMaxDwSplits = 1024;
constexpr int kDwTargetBlocks = 4 * 152;
int64_t dw_tiles(const Net& n, int l) {
  return (int64_t)ceil_div(n.out_dim[l], GT) * ceil_div(n.in_dim[l], GT);
}
// One-row layers go to simt_dw_row_kernel (one block per split, kRowMinPoints or more each).
int splits_for(const Net& n, int l, int64_t npts) {
  const bool row = n.out_dim[l] == 1;
  int64_t S = row ? kMaxDwSplits : ceil_div(kDwTargetBlocks, dw_tiles(n, l));
  S = std::min<int64_t>(S, ceil_div(npts, row ? kRowMinPoints : 2 * GK));
  S = std::min<int64_t>(S, kMaxDwSplits);
  return (int)std::max<int64_t>(S, 1);
}

size_t vjp_layout(const Net& n, int64_t chunk, void* ws, size_t cap, VjpWs* out, bool* ok) {
  Carver c(ws, cap);
  LayerOffs lo;
  VjpWs w;
  w.Wt = c.take<float>(wt_layout(n, &lo));
  w.E = c.take<float>(chunk * n.K0);
  w.Z = c.take<float>(chunk * n.L * n.W);
  w.D = c.take<float>(chunk * n.L * n.W);
  w.dout = c.take<float>(chunk);
  w.f = c.take<float>(chunk);
  // partials of the largest layer at its split count (split counts grow with the chunk)
  int64_t pe = 0;
  for (int l = 0; l <= n.L; ++l)
    pe = std::max<int64_t>(pe, (int64_t)n.out_dim[l] * (n.in_dim[l] + 1) * splits_for(n, l, chunk));
  w.part = c.take<float>(pe);
  if (out) *out = w;
  if (ok) *ok = c.ok;
  return c.off + 256;
}

int prep_wt(const Net& n, const float* theta, float* Wt, LayerOffs* lo, cudaStream_t st) {
  wt_layout(n, lo);
  for (int l = 0; l < n.L; ++l) {
    const int64_t cnt = (int64_t)n.in_dim[l] * n.out_dim[l];
    transpose_w_kernel<<<ceil_div(cnt, 256), 256, 0, st>>>(theta, n.offW[l], n.out_dim[l],
                                                          n.in_dim[l], Wt + lo->Wt[l]);
    INRCT_CHECK_LAUNCH("weight transpose");
  }
  return INRCT_OK;
}

size_t fwd_smem(const Net& n) {
  const int Kmax = n.K0 > n.W ? n.K0 : n.W;
  return sizeof(float) * TP * (Kmax + n.W);
}

int set_fwd_smem(const Net& n) {
  const size_t sm = fwd_smem(n);
  if (sm > 40 * 1024) {  // dynamic plus static shared memory may exceed the 48 KB default
    cudaError_t e = cudaFuncSetAttribute(simt_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) {
      set_error("simt forward smem attribute: %s", cudaGetErrorString(e));
      return INRCT_ERR_CUDA;
    }
  }
  return INRCT_OK;
}

}  // namespace

size_t simt_eval_ws_bytes(const Net& n) {
  LayerOffs lo;
  return align_up(sizeof(float) * wt_layout(n, &lo), 256) + 256;
}

// The hash gather reads both features of a vertex in one 8-byte load.
int check_theta_alignment(const Net& n, const float* theta, const char* who) {
  if (n.kind == INRCT_HASH && (reinterpret_cast<uintptr_t>(theta) & 7) != 0) {
    set_error("%s: theta must be 8-byte aligned for the hash-encoded INR", who);
    return INRCT_ERR_INVALID_ARG;
  }
  return INRCT_OK;
}

int simt_eval(const Net& n, const float* theta, int N, int64_t npts, float* image, void* ws,
              size_t ws_bytes, cudaStream_t st) {
  INRCT_TRY(check_theta_alignment(n, theta, "inr_eval_grid"));
  const size_t need = simt_eval_ws_bytes(n);
  if (!ws || ws_bytes < need) {
    set_error("inr_eval_grid (fp32): workspace of %zu bytes too small (need %zu)", ws_bytes, need);
    return INRCT_ERR_WORKSPACE;
  }
  LayerOffs lo;
  float* Wt = static_cast<float*>(ws);
  INRCT_TRY(prep_wt(n, theta, Wt, &lo, st));
  INRCT_TRY(set_fwd_smem(n));
  prof_mark(kMarkEvalKernel, st);
  simt_fwd_kernel<<<ceil_div(npts, TP), n.W, fwd_smem(n), st>>>(dev_of(n, N), lo, theta, Wt, npts,
                                                               nullptr, image, nullptr, nullptr);
  INRCT_CHECK_LAUNCH("simt forward");
  prof_mark(kMarkEvalDone, st);
  return INRCT_OK;
}

size_t simt_vjp_ws_bytes(const Net& n, int64_t n_idx) {
  const int64_t chunk = n_idx < kVjpChunk ? n_idx : kVjpChunk;
  return vjp_layout(n, chunk, nullptr, 0, nullptr, nullptr);
}

int simt_vjp(const Net& n, const float* theta, int N, const int32_t* idx, int64_t n_idx,
             const float* v, double scale, double* grad_f64, float* grad_f32, double* value_out,
             void* ws, size_t ws_bytes, cudaStream_t st) {
  INRCT_TRY(check_theta_alignment(n, theta, "inr_weighted_vjp"));
  const int64_t chunk = n_idx < kVjpChunk ? n_idx : kVjpChunk;
  VjpWs w;
  bool ok;
  const size_t need = vjp_layout(n, chunk, ws, ws_bytes, &w, &ok);
  if (!ws || !ok) {
    set_error("inr_weighted_vjp (fp32): workspace of %zu bytes too small (need %zu)", ws_bytes, need);
    return INRCT_ERR_WORKSPACE;
  }
  LayerOffs lo;
  INRCT_TRY(prep_wt(n, theta, w.Wt, &lo, st));
  INRCT_TRY(set_fwd_smem(n));
  const NetDev nd = dev_of(n, N);
  for (int64_t c0 = 0; c0 < n_idx; c0 += chunk) {
    const int64_t np = std::min(chunk, n_idx - c0);
    const int32_t* id = idx + c0;
    const unsigned nb = ceil_div(np, TP);
    if (c0 == 0) prof_mark(kMarkVjpKernel, st);
    simt_fwd_kernel<<<nb, n.W, fwd_smem(n), st>>>(nd, lo, theta, w.Wt, np, id, value_out ? w.f : nullptr, w.E,
                                                  w.Z);
    INRCT_CHECK_LAUNCH("simt vjp forward");
    if (c0 == 0 && n.n_table > 0) {
      const cudaError_t e = cudaMemsetAsync(grad_f64, 0, sizeof(double) * n.n_table, st);
      if (e != cudaSuccess) {
        set_error("hash table gradient clear: %s", cudaGetErrorString(e));
        return INRCT_ERR_CUDA;
      }
    }
    simt_bwd_kernel<<<nb, n.W, sizeof(float) * TP * n.W, st>>>(
        nd, lo, theta, np, id, v, (float)scale, w.Z, w.D, w.dout, n.n_table > 0 ? grad_f64 : nullptr);
    INRCT_CHECK_LAUNCH("simt vjp backward");
    if (value_out) {
      weighted_sum_kernel<<<1, 256, 0, st>>>(w.dout, w.f, np, c0 > 0, value_out);
      INRCT_CHECK_LAUNCH("virtual loss sum");
    }
    if (c0 == 0) prof_mark(kMarkVjpKernelDone, st);
    for (int l = 0; l <= n.L; ++l) {
      const int O = n.out_dim[l], K = n.in_dim[l];
      const int S = splits_for(n, l, np);
      const int64_t per = (np + S - 1) / S;
      const float* X = l < n.L ? w.D + (int64_t)l * np * n.W : w.dout;
      const float* Y;
      int ymode;
      if (l == 0) {
        Y = w.E;
        ymode = 0;
      } else {
        Y = w.Z + (int64_t)(l - 1) * np * n.W;
        ymode = n.kind == INRCT_SIREN ? 2 : 1;
      }
      if (O == 1) {
        simt_dw_row_kernel<<<S, (K + 1 + 31) / 32 * 32, 0, st>>>(X, Y, K, ymode, n.omega0, np, per, w.part);
      } else {
        dim3 grd(ceil_div(O, GT), ceil_div(K, GT), S);
        simt_dw_kernel<<<grd, 256, 0, st>>>(X, O, Y, K, ymode, n.omega0, np, per, w.part);
      }
      INRCT_CHECK_LAUNCH("simt dW");
      const int64_t ent = (int64_t)O * (K + 1);
      reduce_layer_kernel<<<ceil_div(ent, 32), 32 * kRedWarps, 0, st>>>(w.part, S, O, K, n.offW[l], n.offb[l],
                                                              1.0, c0 > 0, grad_f64);
      INRCT_CHECK_LAUNCH("simt reduce");
    }
  }
  if (grad_f32) INRCT_TRY(f64_to_f32(grad_f64, grad_f32, n.p, st));
  return INRCT_OK;
}

}  // namespace inrct
