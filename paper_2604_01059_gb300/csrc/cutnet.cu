// CUDA kernels of the cut-order network (training and inference).  The
// network is small (hidden width 64) and its graphs have 10^1..10^2 nodes, so
// each dense layer is a [nodes x K] x [K x 64] product with K <= 128: the
// weights of a layer are staged once per block in shared memory (BF16 values
// widened to FP32), node tiles stream through, and every product accumulates
// in FP32.  Weight gradients are reduced per block into a partial buffer and
// summed in a fixed order, so training is deterministic for a given seed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "cutnet.h"
#include "program.h"
#include "zx.h"

namespace tsim {
namespace cutnet {
namespace {

constexpr int F = kCutFeatures;
constexpr int H = kHidden;
constexpr int OFF_L = (F + 1) * H;     // after [W_in | b_in]
constexpr int LSZ = (2 * H + 1) * H;   // [Ws | Wn | b]
constexpr int OFF_WO = OFF_L + kLayers * LSZ;
constexpr int NPARAM = OFF_WO + H + 1;

constexpr int kThreads = 256;
constexpr int kTile = 32;              // nodes per tile of the dense kernels
constexpr int kMaxK = 2 * H;           // widest input of a dense layer
constexpr int kWgradR = ((kMaxK + 1) * H + kThreads - 1) / kThreads;  // outputs per thread

#define CN_CK(x)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) fail(TSIM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// out[n][c] = act(sum_k A[n][k] Wm[k][c] + bias[c]) over nodes [n0, n1), where
// A = [A1 | A2] (K1 + K2 columns) and Wm = [W1; W2].  TRANS: W1 is a 64 x 64
// matrix used transposed (Wm[k][c] = W1[c][k]), K1 = 64, no A2 and no bias.
template <bool TRANS, bool RELU>
__global__ void __launch_bounds__(kThreads) k_dense(int n0, int n1, const float* __restrict__ A1, int K1,
                                                     const __nv_bfloat16* __restrict__ W1,
                                                     const float* __restrict__ A2, int K2,
                                                     const __nv_bfloat16* __restrict__ W2,
                                                     const __nv_bfloat16* __restrict__ bias,
                                                     float* __restrict__ out) {
  __shared__ float Ws[kMaxK][H];
  __shared__ float As[kTile][kMaxK];
  const int K = K1 + K2;
  for (int i = threadIdx.x; i < K * H; i += kThreads) {
    const int k = i / H, c = i % H;
    float w;
    if (TRANS) w = __bfloat162float(W1[c * H + k]);
    else w = k < K1 ? __bfloat162float(W1[k * H + c]) : __bfloat162float(W2[(k - K1) * H + c]);
    Ws[k][c] = w;
  }
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  float b[4];
  for (int c = 0; c < 4; ++c) b[c] = bias ? __bfloat162float(bias[tx + 16 * c]) : 0.0f;
  for (int base = n0 + blockIdx.x * kTile; base < n1; base += gridDim.x * kTile) {
    __syncthreads();  // Ws ready / previous tile consumed
    for (int i = threadIdx.x; i < kTile * K; i += kThreads) {
      const int r = i / K, k = i % K, node = base + r;
      float a = 0.0f;
      if (node < n1) a = k < K1 ? A1[(size_t)node * K1 + k] : A2[(size_t)node * K2 + (k - K1)];
      As[r][k] = a;
    }
    __syncthreads();
    float acc[2][4];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 4; ++c) acc[r][c] = b[c];
    for (int k = 0; k < K; ++k) {
      const float a0 = As[2 * ty][k], a1 = As[2 * ty + 1][k];
      for (int c = 0; c < 4; ++c) {
        const float w = Ws[k][tx + 16 * c];
        acc[0][c] = fmaf(a0, w, acc[0][c]);
        acc[1][c] = fmaf(a1, w, acc[1][c]);
      }
    }
    for (int r = 0; r < 2; ++r) {
      const int node = base + 2 * ty + r;
      if (node >= n1) continue;
      for (int c = 0; c < 4; ++c) {
        float v = acc[r][c];
        if (RELU) v = fmaxf(v, 0.0f);
        out[(size_t)node * H + tx + 16 * c] = v;
      }
    }
  }
}

// M[v] = mean of Hin[u] over the neighbours u of v (16 threads per node, 4 features each)
__global__ void k_agg_fwd(int n0, int n1, const int* __restrict__ rowptr, const int* __restrict__ col,
                          const float4* __restrict__ Hin, float4* __restrict__ M) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int v = n0 + (int)(t / 16), q = (int)(t % 16);
  if (v >= n1) return;
  const int e0 = rowptr[v], e1 = rowptr[v + 1];
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e = e0; e < e1; ++e) {
    const float4 h = Hin[(size_t)col[e] * 16 + q];
    s.x += h.x; s.y += h.y; s.z += h.z; s.w += h.w;
  }
  const float inv = e1 > e0 ? 1.0f / (float)(e1 - e0) : 0.0f;
  M[(size_t)v * 16 + q] = make_float4(s.x * inv, s.y * inv, s.z * inv, s.w * inv);
}

// out[u] = (D[u] + sum over neighbours v of G[v] / deg(v)) masked by Hmask[u] > 0:
// the gradient through the mean aggregation (the adjacency is symmetric) and
// the ReLU that produced Hmask.
__global__ void k_agg_bwd(int n0, int n1, const int* __restrict__ rowptr, const int* __restrict__ col,
                          const float4* __restrict__ G, const float4* __restrict__ D,
                          const float4* __restrict__ Hmask, float4* __restrict__ out) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int u = n0 + (int)(t / 16), q = (int)(t % 16);
  if (u >= n1) return;
  float4 s = D[(size_t)u * 16 + q];
  for (int e = rowptr[u]; e < rowptr[u + 1]; ++e) {
    const int v = col[e];
    const float inv = 1.0f / (float)(rowptr[v + 1] - rowptr[v]);
    const float4 g = G[(size_t)v * 16 + q];
    s.x = fmaf(g.x, inv, s.x); s.y = fmaf(g.y, inv, s.y);
    s.z = fmaf(g.z, inv, s.z); s.w = fmaf(g.w, inv, s.w);
  }
  const float4 m = Hmask[(size_t)u * 16 + q];
  out[(size_t)u * 16 + q] = make_float4(m.x > 0.f ? s.x : 0.f, m.y > 0.f ? s.y : 0.f,
                                        m.z > 0.f ? s.z : 0.f, m.w > 0.f ? s.w : 0.f);
}

// s[v] = H3[v] . w_o + b_o, one warp per node
__global__ void k_head(int n0, int n1, const float* __restrict__ H3, const __nv_bfloat16* __restrict__ wo,
                       float* __restrict__ s) {
  const int lane = threadIdx.x & 31;
  const int v = n0 + (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (v >= n1) return;
  float acc = H3[(size_t)v * H + lane] * __bfloat162float(wo[lane]);
  acc = fmaf(H3[(size_t)v * H + lane + 32], __bfloat162float(wo[lane + 32]), acc);
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) s[v] = acc + __bfloat162float(wo[H]);
}

// dZ3[v][j] = ds[v] w_o[j], masked by H3[v][j] > 0
__global__ void k_head_bwd(int n0, int n1, const float* __restrict__ ds, const __nv_bfloat16* __restrict__ wo,
                           const float* __restrict__ H3, float* __restrict__ dZ) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int v = n0 + (int)(t / H), j = (int)(t % H);
  if (v >= n1) return;
  const size_t i = (size_t)v * H + j;
  dZ[i] = H3[i] > 0.f ? ds[v] * __bfloat162float(wo[j]) : 0.0f;
}

// Per-graph centred squared error (block per graph): gl[g] = mean over the
// labelled nodes of d^2, ds[v] = 2 d_v inv_G / |L_g|, d = centred(s) - centred(y).
__global__ void k_loss(int g0, const int* __restrict__ goff, const float* __restrict__ s,
                       const float* __restrict__ y, float inv_G, float* __restrict__ ds, float* __restrict__ gl) {
  const int g = g0 + blockIdx.x;
  const int a = goff[g], b = goff[g + 1];
  __shared__ float red[3][32];
  float cnt = 0.f, ss = 0.f, sy = 0.f;
  for (int v = a + threadIdx.x; v < b; v += blockDim.x)
    if (!isnan(y[v])) { cnt += 1.f; ss += s[v]; sy += y[v]; }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o; o >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  if (lane == 0) { red[0][w] = cnt; red[1][w] = ss; red[2][w] = sy; }
  __syncthreads();
  cnt = ss = sy = 0.f;
  for (int i = 0; i < nw; ++i) { cnt += red[0][i]; ss += red[1][i]; sy += red[2][i]; }
  __syncthreads();
  const bool use = cnt >= 2.f;
  const float ms = use ? ss / cnt : 0.f, my = use ? sy / cnt : 0.f;
  float l = 0.f;
  for (int v = a + threadIdx.x; v < b; v += blockDim.x) {
    float gv = 0.f;
    if (use && !isnan(y[v])) {
      const float d = (s[v] - ms) - (y[v] - my);
      l = fmaf(d, d, l);
      gv = 2.f * d * inv_G / cnt;
    }
    ds[v] = gv;
  }
  for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if (lane == 0) red[0][w] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < nw; ++i) t += red[0][i];
    gl[g] = use ? t / cnt : 0.f;
  }
}

// Weight gradient of one layer: partial[blk][k][j] = sum over the block's
// nodes of A[n][k] G[n][j], with A = [A1 | A2 | 1] (the ones column gives the
// bias row).  Output o = k * J + j is owned by thread o mod 256.
__global__ void __launch_bounds__(kThreads) k_wgrad(int n0, int n1, int chunk, const float* __restrict__ A1, int K1,
                                                     const float* __restrict__ A2, int K2,
                                                     const float* __restrict__ G, int J,
                                                     float* __restrict__ partial) {
  __shared__ float As[kTile][kMaxK + 1];
  __shared__ float Gs[kTile][H];
  const int K = K1 + K2, O = (K + 1) * J;
  const int lo = n0 + blockIdx.x * chunk, hi = min(n1, lo + chunk);
  float acc[kWgradR];
  int kk[kWgradR], jj[kWgradR];
#pragma unroll
  for (int r = 0; r < kWgradR; ++r) {
    acc[r] = 0.f;
    const int o = threadIdx.x + kThreads * r;
    kk[r] = o < O ? o / J : K + 1;
    jj[r] = o < O ? o % J : 0;
  }
  for (int base = lo; base < hi; base += kTile) {
    __syncthreads();
    for (int i = threadIdx.x; i < kTile * (K + 1); i += kThreads) {
      const int r = i / (K + 1), k = i % (K + 1), node = base + r;
      float a = 0.f;
      if (node < hi) a = k < K1 ? A1[(size_t)node * K1 + k] : (k < K ? A2[(size_t)node * K2 + (k - K1)] : 1.f);
      As[r][k] = a;
    }
    for (int i = threadIdx.x; i < kTile * J; i += kThreads) {
      const int r = i / J, j = i % J, node = base + r;
      Gs[r][j] = node < hi ? G[(size_t)node * J + j] : 0.f;
    }
    __syncthreads();
    for (int n = 0; n < kTile; ++n) {
#pragma unroll
      for (int r = 0; r < kWgradR; ++r)
        if (kk[r] <= K) acc[r] = fmaf(As[n][kk[r]], Gs[n][jj[r]], acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < kWgradR; ++r) {
    const int o = threadIdx.x + kThreads * r;
    if (o < O) partial[(size_t)blockIdx.x * O + o] = acc[r];
  }
}

// grad[o] = sum over blocks of partial[b][o], in block order
__global__ void k_reduce(const float* __restrict__ partial, int nblk, int O, float* __restrict__ grad) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= O) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * O + o];
  grad[o] = s;
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ w, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = __float2bfloat16_rn(p[i]);
}

// Adam constants for step t (beta1 0.9, beta2 0.999, eps 1e-8): the
// complements 1 - beta and the bias corrections 1 - beta^t are formed in
// double and rounded once (1 - 0.999f in float would be 1.3e-5 off 0.001).
struct AdamConsts {
  float b1, omb1, b2, omb2, eps, bc1, bc2;
};

AdamConsts adam_consts(int step) {
  const double b1 = 0.9, b2 = 0.999;
  return {(float)b1, (float)(1.0 - b1), (float)b2, (float)(1.0 - b2), 1e-8f,
          (float)(1.0 - std::pow(b1, (double)step)), (float)(1.0 - std::pow(b2, (double)step))};
}

// Adam (Kingma and Ba, 2015) on the FP32 master copy; refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ w, int n, float lr, AdamConsts k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = k.b1 * m[i] + k.omb1 * gi;
  const float vi = k.b2 * v[i] + k.omb2 * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / k.bc1) / (sqrtf(vi / k.bc2) + k.eps);
  p[i] = pi;
  w[i] = __float2bfloat16_rn(pi);
}

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  void ensure(size_t want) {
    if (want <= n) return;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    CN_CK(cudaMalloc(&p, std::max<size_t>(want, 1) * sizeof(T)));
    n = want;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

// Device state of one network: parameters, activations of a node range,
// gradients and optimiser state.
struct Net {
  DevBuf<float> P, G, Mo, Vo, partial;
  DevBuf<__nv_bfloat16> Wb;
  DevBuf<float> X, Hs[kLayers + 1], Ms[kLayers], s, ds, gl, dZa, dZb, D, Gn, y;
  DevBuf<int> rowptr, col, goff;
  cudaStream_t st = nullptr;
  int max_blocks = 0;  // two blocks per SM of the current device

  int blocks_cap() {
    if (!max_blocks) {
      int dev = 0, sms = 0;
      CN_CK(cudaGetDevice(&dev));
      CN_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      max_blocks = 2 * std::max(1, sms);
    }
    return max_blocks;
  }

  void release() {
    max_blocks = 0;
    for (DevBuf<float>* b : {&P, &G, &Mo, &Vo, &partial, &X, &s, &ds, &gl, &dZa, &dZb, &D, &Gn, &y}) b->release();
    for (auto& b : Hs) b.release();
    for (auto& b : Ms) b.release();
    Wb.release();
    rowptr.release();
    col.release();
    goff.release();
  }

  void upload_params(const float* params) {
    P.ensure(NPARAM);
    Wb.ensure(NPARAM);
    CN_CK(cudaMemcpyAsync(P.p, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice, st));
    k_to_bf16<<<(NPARAM + 255) / 256, 256, 0, st>>>(P.p, Wb.p, NPARAM);
    CN_CK(cudaGetLastError());
  }

  void upload_graphs(const Batch& b) {
    const size_t n = (size_t)b.n;
    if (b.X.size() != n * F || b.rowptr.size() != n + 1 || b.goff.empty())
      fail(TSIM_ERR_ARG, "inconsistent graph batch");
    X.ensure(n * F);
    rowptr.ensure(n + 1);
    col.ensure(b.col.size());
    goff.ensure(b.goff.size());
    for (auto& h : Hs) h.ensure(n * H);
    for (auto& m : Ms) m.ensure(n * H);
    s.ensure(n);
    if (n) CN_CK(cudaMemcpyAsync(X.p, b.X.data(), n * F * sizeof(float), cudaMemcpyHostToDevice, st));
    CN_CK(cudaMemcpyAsync(rowptr.p, b.rowptr.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    if (!b.col.empty())
      CN_CK(cudaMemcpyAsync(col.p, b.col.data(), b.col.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CN_CK(cudaMemcpyAsync(goff.p, b.goff.data(), b.goff.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  }

  void alloc_training(const Batch& b) {
    const size_t n = (size_t)b.n;
    G.ensure(NPARAM);
    ds.ensure(n);
    gl.ensure(b.goff.size());
    dZa.ensure(n * H);
    dZb.ensure(n * H);
    D.ensure(n * H);
    Gn.ensure(n * H);
    y.ensure(n);
    partial.ensure((size_t)blocks_cap() * (kMaxK + 1) * H);
    if (n) CN_CK(cudaMemcpyAsync(y.p, b.y.data(), n * sizeof(float), cudaMemcpyHostToDevice, st));
  }

  int dense_blocks(int n) { return std::max(1, std::min(blocks_cap(), (n + kTile - 1) / kTile)); }
  static int node_blocks(long threads) { return (int)std::max(1L, (threads + 255) / 256); }

  const __nv_bfloat16* w(int off) const { return Wb.p + off; }

  void forward(int n0, int n1) {
    const int n = n1 - n0;
    if (n <= 0) return;
    const int db = dense_blocks(n);
    k_dense<false, true><<<db, kThreads, 0, st>>>(n0, n1, X.p, F, w(0), nullptr, 0, nullptr, w(F * H), Hs[0].p);
    for (int l = 0; l < kLayers; ++l) {
      const int off = OFF_L + l * LSZ;
      k_agg_fwd<<<node_blocks(16L * n), 256, 0, st>>>(n0, n1, rowptr.p, col.p, (const float4*)Hs[l].p,
                                                       (float4*)Ms[l].p);
      k_dense<false, true><<<db, kThreads, 0, st>>>(n0, n1, Hs[l].p, H, w(off), Ms[l].p, H, w(off + H * H),
                                                     w(off + 2 * H * H), Hs[l + 1].p);
    }
    k_head<<<node_blocks(32L * n), 256, 0, st>>>(n0, n1, Hs[kLayers].p, w(OFF_WO), s.p);
    CN_CK(cudaGetLastError());
  }

  void wgrad(int n0, int n1, const float* A1, int K1, const float* A2, int K2, const float* Gd, int J, int off) {
    const int n = n1 - n0;
    const int nblk = std::max(1, std::min(blocks_cap(), (n + 63) / 64));
    const int chunk = (n + nblk - 1) / nblk;
    const int O = (K1 + K2 + 1) * J;
    k_wgrad<<<nblk, kThreads, 0, st>>>(n0, n1, chunk, A1, K1, A2, K2, Gd, J, partial.p);
    k_reduce<<<(O + 255) / 256, 256, 0, st>>>(partial.p, nblk, O, G.p + off);
  }

  // loss of graphs [g0, g1) (nodes goff[g0]..goff[g1]); gradient into G
  void backward(int g0, int g1, int n0, int n1, float inv_G) {
    const int n = n1 - n0;
    if (g1 > g0) k_loss<<<g1 - g0, 128, 0, st>>>(g0, goff.p, s.p, y.p, inv_G, ds.p, gl.p);
    CN_CK(cudaMemsetAsync(G.p, 0, NPARAM * sizeof(float), st));
    if (n <= 0) return;
    const int db = dense_blocks(n);
    wgrad(n0, n1, Hs[kLayers].p, H, nullptr, 0, ds.p, 1, OFF_WO);
    k_head_bwd<<<node_blocks((long)H * n), 256, 0, st>>>(n0, n1, ds.p, w(OFF_WO), Hs[kLayers].p, dZa.p);
    float* dZ = dZa.p;      // gradient at the pre-activation of H_{l+1}
    float* dZn = dZb.p;
    for (int l = kLayers - 1; l >= 0; --l) {
      const int off = OFF_L + l * LSZ;
      wgrad(n0, n1, Hs[l].p, H, Ms[l].p, H, dZ, H, off);
      k_dense<true, false><<<db, kThreads, 0, st>>>(n0, n1, dZ, H, w(off), nullptr, 0, nullptr, nullptr, D.p);
      k_dense<true, false><<<db, kThreads, 0, st>>>(n0, n1, dZ, H, w(off + H * H), nullptr, 0, nullptr, nullptr,
                                                     Gn.p);
      k_agg_bwd<<<node_blocks(16L * n), 256, 0, st>>>(n0, n1, rowptr.p, col.p, (const float4*)Gn.p,
                                                       (const float4*)D.p, (const float4*)Hs[l].p, (float4*)dZn);
      std::swap(dZ, dZn);
    }
    wgrad(n0, n1, X.p, F, nullptr, 0, dZ, H, 0);
    CN_CK(cudaGetLastError());
  }
};

float inv_graph_count(const Batch& b, int g0, int g1) {
  int cnt = 0;
  for (int g = g0; g < g1; ++g) {
    int l = 0;
    for (int v = b.goff[(size_t)g]; v < b.goff[(size_t)g + 1]; ++v) l += !std::isnan(b.y[(size_t)v]);
    cnt += l >= 2;
  }
  return cnt ? 1.0f / (float)cnt : 0.0f;
}

struct StreamGuard {
  cudaStream_t s = nullptr;
  StreamGuard() { CN_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)); }
  ~StreamGuard() {
    if (s) cudaStreamDestroy(s);
  }
};

struct NetGuard {
  Net net;
  StreamGuard sg;
  NetGuard() { net.st = sg.s; }
  ~NetGuard() {
    cudaStreamSynchronize(net.st);
    net.release();
  }
};

// the registered scorer: parameters stay on the device between calls
std::mutex g_model_mu;
Net* g_model = nullptr;
cudaStream_t g_model_stream = nullptr;
int g_model_device = -1;

bool gpu_scorer(const Graph& g, std::vector<double>& scores) {
  Batch b;
  std::vector<int> uids;
  cut_features(g, b.X, b.rowptr, b.col, uids);
  b.n = (int)uids.size();
  b.goff = {0, b.n};
  std::vector<float> s((size_t)b.n);
  try {
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (!g_model) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g_model_device) return false;
    g_model->upload_graphs(b);
    g_model->forward(0, b.n);
    if (b.n)
      CN_CK(cudaMemcpyAsync(s.data(), g_model->s.p, (size_t)b.n * sizeof(float), cudaMemcpyDeviceToHost,
                            g_model->st));
    CN_CK(cudaStreamSynchronize(g_model->st));
  } catch (const Error&) {
    return false;
  }
  int mx = -1;
  for (int u : uids) mx = std::max(mx, u);
  scores.assign((size_t)(mx + 1), 1e300);
  for (size_t i = 0; i < uids.size(); ++i)
    if (uids[i] >= 0) scores[(size_t)uids[i]] = s[i];
  return true;
}

}  // namespace

int num_params() { return NPARAM; }

void init_params(uint64_t seed, float* p) {
  // uniform(-sqrt(6/fan_in), +sqrt(6/fan_in)) weights (He et al., 2015),
  // zero biases, from a splitmix64 stream
  uint64_t st = seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
  auto uni = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  };
  std::fill(p, p + NPARAM, 0.0f);
  const double bin = std::sqrt(6.0 / F);
  for (int i = 0; i < F * H; ++i) p[i] = (float)(bin * uni());
  const double bh = std::sqrt(6.0 / (2 * H));
  for (int l = 0; l < kLayers; ++l)
    for (int i = 0; i < 2 * H * H; ++i) p[OFF_L + l * LSZ + i] = (float)(bh * uni());
  const double bo = std::sqrt(3.0 / H);
  for (int i = 0; i < H; ++i) p[OFF_WO + i] = (float)(bo * uni());
}

void forward(const float* params, const Batch& b, float* scores) {
  NetGuard ng;
  Net& net = ng.net;
  net.upload_params(params);
  net.upload_graphs(b);
  net.forward(0, b.n);
  if (b.n) CN_CK(cudaMemcpyAsync(scores, net.s.p, (size_t)b.n * sizeof(float), cudaMemcpyDeviceToHost, net.st));
  CN_CK(cudaStreamSynchronize(net.st));
}

double loss_grad(const float* params, const Batch& b, float* grad) {
  NetGuard ng;
  Net& net = ng.net;
  const int G = (int)b.goff.size() - 1;
  net.upload_params(params);
  net.upload_graphs(b);
  net.alloc_training(b);
  net.forward(0, b.n);
  net.backward(0, G, 0, b.n, inv_graph_count(b, 0, G));
  std::vector<float> gl((size_t)std::max(G, 0));
  CN_CK(cudaMemcpyAsync(grad, net.G.p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, net.st));
  if (G) CN_CK(cudaMemcpyAsync(gl.data(), net.gl.p, (size_t)G * sizeof(float), cudaMemcpyDeviceToHost, net.st));
  CN_CK(cudaStreamSynchronize(net.st));
  const float ig = inv_graph_count(b, 0, G);
  double loss = 0.0;
  for (float x : gl) loss += x;
  return loss * ig;
}

void adam_step(float* params, const float* grad, float* m, float* v, int n, int step, float lr) {
  if (n != NPARAM || step < 1) fail(TSIM_ERR_ARG, "adam_step: bad size or step");
  NetGuard ng;
  Net& net = ng.net;
  net.P.ensure(NPARAM);
  net.G.ensure(NPARAM);
  net.Mo.ensure(NPARAM);
  net.Vo.ensure(NPARAM);
  net.Wb.ensure(NPARAM);
  const size_t by = NPARAM * sizeof(float);
  CN_CK(cudaMemcpyAsync(net.P.p, params, by, cudaMemcpyHostToDevice, net.st));
  CN_CK(cudaMemcpyAsync(net.G.p, grad, by, cudaMemcpyHostToDevice, net.st));
  CN_CK(cudaMemcpyAsync(net.Mo.p, m, by, cudaMemcpyHostToDevice, net.st));
  CN_CK(cudaMemcpyAsync(net.Vo.p, v, by, cudaMemcpyHostToDevice, net.st));
  k_adam<<<(NPARAM + 255) / 256, 256, 0, net.st>>>(net.P.p, net.G.p, net.Mo.p, net.Vo.p, net.Wb.p, NPARAM, lr,
                                                   adam_consts(step));
  CN_CK(cudaGetLastError());
  CN_CK(cudaMemcpyAsync(params, net.P.p, by, cudaMemcpyDeviceToHost, net.st));
  CN_CK(cudaMemcpyAsync(m, net.Mo.p, by, cudaMemcpyDeviceToHost, net.st));
  CN_CK(cudaMemcpyAsync(v, net.Vo.p, by, cudaMemcpyDeviceToHost, net.st));
  CN_CK(cudaStreamSynchronize(net.st));
}

void train(const Batch& b, int epochs, int batch_graphs, float lr, uint64_t seed, float* params,
           float* loss_per_epoch) {
  const int G = (int)b.goff.size() - 1;
  if (epochs < 1 || batch_graphs < 1 || G < 1 || !(lr > 0.0f)) fail(TSIM_ERR_ARG, "bad training parameters");
  NetGuard ng;
  Net& net = ng.net;
  net.upload_params(params);
  net.upload_graphs(b);
  net.alloc_training(b);
  net.Mo.ensure(NPARAM);
  net.Vo.ensure(NPARAM);
  CN_CK(cudaMemsetAsync(net.Mo.p, 0, NPARAM * sizeof(float), net.st));
  CN_CK(cudaMemsetAsync(net.Vo.p, 0, NPARAM * sizeof(float), net.st));
  const int nb = (G + batch_graphs - 1) / batch_graphs;
  std::vector<int> order((size_t)nb);
  std::vector<float> invg((size_t)nb);
  for (int i = 0; i < nb; ++i) {
    order[(size_t)i] = i;
    invg[(size_t)i] = inv_graph_count(b, i * batch_graphs, std::min(G, (i + 1) * batch_graphs));
  }
  uint64_t st = seed ^ 0xA0761D6478BD642Full;
  auto rnd = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  std::vector<float> gl((size_t)G);
  int step = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (size_t i = order.size(); i > 1; --i) std::swap(order[i - 1], order[(size_t)(rnd() % i)]);
    for (int bi : order) {
      const int g0 = bi * batch_graphs, g1 = std::min(G, g0 + batch_graphs);
      const int n0 = b.goff[(size_t)g0], n1 = b.goff[(size_t)g1];
      net.forward(n0, n1);
      net.backward(g0, g1, n0, n1, invg[(size_t)bi]);
      ++step;
      k_adam<<<(NPARAM + 255) / 256, 256, 0, net.st>>>(net.P.p, net.G.p, net.Mo.p, net.Vo.p, net.Wb.p, NPARAM, lr,
                                                       adam_consts(step));
      CN_CK(cudaGetLastError());
    }
    CN_CK(cudaMemcpyAsync(gl.data(), net.gl.p, (size_t)G * sizeof(float), cudaMemcpyDeviceToHost, net.st));
    CN_CK(cudaStreamSynchronize(net.st));
    if (loss_per_epoch) {
      // mean over minibatches of the minibatch loss (each taken before its step)
      double tot = 0.0;
      for (int i = 0; i < nb; ++i) {
        double s = 0.0;
        for (int g = i * batch_graphs; g < std::min(G, (i + 1) * batch_graphs); ++g) s += gl[(size_t)g];
        tot += s * invg[(size_t)i];
      }
      loss_per_epoch[ep] = (float)(tot / nb);
    }
  }
  CN_CK(cudaMemcpyAsync(params, net.P.p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, net.st));
  CN_CK(cudaStreamSynchronize(net.st));
}

void set_model(const float* params) {
  std::lock_guard<std::mutex> lk(g_model_mu);
  g_cut_scorer.store(nullptr);
  if (g_model) {
    if (g_model_stream) cudaStreamSynchronize(g_model_stream);
    g_model->release();
    delete g_model;
    g_model = nullptr;
  }
  if (g_model_stream) {
    cudaStreamDestroy(g_model_stream);
    g_model_stream = nullptr;
  }
  if (!params) return;
  int dev = -1;
  CN_CK(cudaGetDevice(&dev));
  CN_CK(cudaStreamCreateWithFlags(&g_model_stream, cudaStreamNonBlocking));
  g_model = new Net;
  g_model->st = g_model_stream;
  g_model_device = dev;
  g_model->upload_params(params);
  CN_CK(cudaStreamSynchronize(g_model_stream));
  g_cut_scorer.store(&gpu_scorer);
}

}  // namespace cutnet
}  // namespace tsim
