// J-interpolation surrogate network: hand-written training and inference kernels.
//
// Network: n_in inputs -> depth hidden layers of width W with GELU (tanh form) -> 1
// output; weights held in BF16 for the forward and backward products, with FP32 master
// weights and AdamW moments; activations and accumulation in FP32. The network is
// small (4 -> 256 -> 256 -> 256 -> 1 is 133k parameters), so the products run on
// CUDA cores in register-tiled 128 x 64 blocks (8 x 4 outputs per thread) with the
// operand layouts fixed at compile time; the weight gradients, whose contraction runs
// over the batch, are split over the batch into partial products summed in a fixed order.
//
// Parameter order (flat, as exchanged with the host): for each layer l = 0..depth,
// W_l (row-major [out][in]) then b_l.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "../../include/mw3.h"

namespace {

__device__ __forceinline__ float gelu_f(float z) {
  const float s = 0.7978845608028654f, a = 0.044715f;
  return 0.5f * z * (1.0f + tanhf(s * (z + a * z * z * z)));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  const float s = 0.7978845608028654f, a = 0.044715f;
  const float t = tanhf(s * (z + a * z * z * z));
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * s * (1.0f + 3.0f * a * z * z);
}

// C[M x N] = A[M x K] B[K x N] with an epilogue:
//   mode 0: C = acc + bias[n]; Z = C; H = gelu(C) (hidden layer forward)
//   mode 1: C = acc + bias[n] (output layer forward)
//   mode 2: C = acc * gelu'(Z[m][n]) (backward through a hidden activation)
//   mode 3: C = acc (weight gradient)
// The product runs in 128 x 64 tiles, 256 threads,
// each thread 8 rows (8 ty .. 8 ty + 7) x 4 columns (4 tx .. 4 tx + 3) read from shared
// memory as float4. The layouts are template parameters: AT / BT transpose the operand's
// storage (element (r, c) at c * ld + r), AH / BH read the BF16 weight copy. split > 1
// (mode 3 only): CTA z takes rows [z, z + 1) * kchunk of K and writes its partial product
// to C + z * M * ldc (summed afterwards by k_sum_splits in a fixed order).
constexpr int TBM = 128, TBN = 64, TBK = 16, TPAD = 4;

template <bool AT, bool AH, bool BT, bool BH>
__global__ void __launch_bounds__(256) k_mlp_gemm_t(int M, int N, int K, int kchunk,
                                                    const void* __restrict__ Ap, long lda,
                                                    const void* __restrict__ Bp, long ldb,
                                                    float* __restrict__ C, long ldc,
                                                    const float* __restrict__ bias,
                                                    const float* __restrict__ Z,
                                                    float* __restrict__ H, int mode) {
  __shared__ __align__(16) float As[TBK][TBM + TPAD];
  __shared__ __align__(16) float Bs[TBK][TBN + TPAD];
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  auto ldA = [&](long r, long c) -> float {   // A(r, c), r < M, c < K
    const long i = AT ? c * lda + r : r * lda + c;
    if constexpr (AH) return __bfloat162float(static_cast<const __nv_bfloat16*>(Ap)[i]);
    else return static_cast<const float*>(Ap)[i];
  };
  auto ldB = [&](long r, long c) -> float {   // B(r, c), r < K, c < N
    const long i = BT ? c * ldb + r : r * ldb + c;
    if constexpr (BH) return __bfloat162float(static_cast<const __nv_bfloat16*>(Bp)[i]);
    else return static_cast<const float*>(Bp)[i];
  };
  float acc[8][4] = {};
  // the next K tile is read from global memory into registers while the current one is
  // multiplied from shared memory, so the loads overlap the arithmetic
  constexpr int NA = TBM * TBK / 256, NB = TBN * TBK / 256;
  float ra[NA], rb[NB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < NA; ++u) {   // with AT the storage is contiguous along m, else along k
      const int e = tid + 256 * u;
      const int mm = AT ? (e % TBM) : (e / TBK), kk = AT ? (e / TBM) : (e % TBK);
      const int m = m0 + mm, k = k0 + kk;
      ra[u] = (m < M && k < kend) ? ldA(m, k) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int e = tid + 256 * u;
      const int nn = BT ? (e / TBK) : (e % TBN), kk = BT ? (e % TBK) : (e / TBN);
      const int n = n0 + nn, k = k0 + kk;
      rb[u] = (n < N && k < kend) ? ldB(k, n) : 0.0f;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int e = tid + 256 * u;
      const int mm = AT ? (e % TBM) : (e / TBK), kk = AT ? (e / TBM) : (e % TBK);
      As[kk][mm] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int e = tid + 256 * u;
      const int nn = BT ? (e / TBK) : (e % TBN), kk = BT ? (e % TBK) : (e / TBN);
      Bs[kk][nn] = rb[u];
    }
  };
  if (kbeg < kend) fetch(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += TBK) {
    stash();
    __syncthreads();
    if (k0 + TBK < kend) fetch(k0 + TBK);
#pragma unroll
    for (int kk = 0; kk < TBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][8 * ty]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][8 * ty + 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* Cz = C + (long)blockIdx.z * M * ldc;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + 8 * ty + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + 4 * tx + j;
      if (n >= N) continue;
      float v = acc[i][j];
      const long o = (long)m * ldc + n;
      if (mode == 0) {
        v += bias[n];
        C[o] = v;
        H[o] = gelu_f(v);
      } else if (mode == 1) {
        C[o] = v + bias[n];
      } else if (mode == 2) {
        C[o] = v * gelu_grad_f(Z[o]);
      } else {
        Cz[o] = v;
      }
    }
  }
}

// out[e] = sum_z part[z][e], z in order (the split-batch weight gradients)
__global__ void k_sum_splits(const float* __restrict__ part, int nsplit, long n,
                             float* __restrict__ out) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int z = 0; z < nsplit; ++z) s += part[(long)z * n + e];
    out[e] = s;
  }
}

// Gather a minibatch: Xb[r] = X[idx[r]], yb[r] = y[idx[r]]
__global__ void k_gather(const float* __restrict__ X, const float* __restrict__ y,
                         const int* __restrict__ idx, int n, int nin, float* __restrict__ Xb,
                         float* __restrict__ yb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int s = idx[r];
  for (int i = 0; i < nin; ++i) Xb[(long)r * nin + i] = X[(long)s * nin + i];
  yb[r] = y[s];
}

// g[r] = (2/n) (out[r] - y[r]); partial squared errors per block (fixed order)
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ y, int n,
                      float* __restrict__ g, double* __restrict__ partial) {
  __shared__ double red[256];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0;
  if (r < n) {
    const float d = out[r] - y[r];
    g[r] = 2.0f * d / (float)n;
    s = (double)d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// loss[0] = (sum_b partial[b]) / n, the block partials in order (one thread)
__global__ void k_loss_sum(const double* __restrict__ partial, int nb, double n,
                           double* __restrict__ loss) {
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[b];
  *loss = s / n;
}

// db[o] = sum_r g[r][o] in two fixed-order stages: CTA (column tile, row chunk) sums its rows
// with lane = column (coalesced) and warp = row stride 8, the eight warps in order; then the
// chunks in order (k_sum_splits).
constexpr int kColChunk = 512;
__global__ void __launch_bounds__(256) k_colsum_part(const float* __restrict__ g, int n, int nout,
                                                     float* __restrict__ part) {
  __shared__ float red[8][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + lane;
  const int r0 = blockIdx.y * kColChunk, r1 = min(n, r0 + kColChunk);
  float s = 0.0f;
  if (o < nout)
    for (int r = r0 + warp; r < r1; r += 8) s += g[(long)r * nout + o];
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && o < nout) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += red[w][lane];
    part[(long)blockIdx.y * nout + o] = t;
  }
}

// AdamW on FP32 master parameters; refreshes the BF16 copy of weights (wmask = 1).
__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, __nv_bfloat16* __restrict__ ph,
                        const unsigned char* __restrict__ wmask, long n, float lr, float b1,
                        float b2, float eps, float wd, float c1, float c2) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / c1, vh = vi / c2;
  const float decay = wmask[i] ? wd * p[i] : 0.f;
  const float np = p[i] - lr * (mh / (sqrtf(vh) + eps) + decay);
  p[i] = np;
  ph[i] = __float2bfloat16_rn(np);
}

}  // namespace

struct mw3_mlp {
  int device = 0;
  int nin = 4, width = 256, depth = 3;
  std::vector<int> sizes;            // layer widths: nin, W, ..., W, 1
  std::vector<long> woff, boff;      // offsets of W_l and b_l in the flat arrays
  long nparam = 0;
  float* p = nullptr;                // FP32 master parameters
  __nv_bfloat16* ph = nullptr;       // BF16 copy (all parameters; biases unused in BF16)
  float *g = nullptr, *m = nullptr, *v = nullptr;
  unsigned char* wmask = nullptr;    // 1 for weights (decayed), 0 for biases
  long step = 0;
  // activations for a batch of up to cap rows
  long cap = 0;
  std::vector<float*> Zs, Hs, Gs;    // per layer: pre-activation, activation, gradient
  float *X = nullptr, *y = nullptr, *out = nullptr, *gout = nullptr;
  double* partial = nullptr;
  float *Xall = nullptr, *yall = nullptr;
  int* idx = nullptr;
  float* split = nullptr;            // partial weight gradients of the split batch
  long split_cap = 0;
  long nall = 0;
  std::string err;
};

namespace {
int mfail(mw3_mlp* n, int code, const std::string& s) {
  n->err = s;
  return code;
}

#define MCK(call)                                                                             \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return mfail(net, MW3_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void free_acts(mw3_mlp* net) {
  for (auto* p : net->Zs) cudaFree(p);
  for (auto* p : net->Hs) cudaFree(p);
  for (auto* p : net->Gs) cudaFree(p);
  net->Zs.clear();
  net->Hs.clear();
  net->Gs.clear();
  cudaFree(net->X);
  cudaFree(net->y);
  cudaFree(net->out);
  cudaFree(net->gout);
  cudaFree(net->partial);
  net->X = net->y = net->out = net->gout = nullptr;
  net->partial = nullptr;
  net->cap = 0;
}

int ensure_cap(mw3_mlp* net, long rows) {
  if (rows <= net->cap) return MW3_OK;
  free_acts(net);
  const int L = (int)net->sizes.size() - 1;
  for (int l = 0; l < L; ++l) {
    float *z, *h, *g;
    MCK(cudaMalloc(&z, rows * net->sizes[l + 1] * sizeof(float)));
    MCK(cudaMalloc(&h, rows * net->sizes[l + 1] * sizeof(float)));
    MCK(cudaMalloc(&g, rows * net->sizes[l + 1] * sizeof(float)));
    net->Zs.push_back(z);
    net->Hs.push_back(h);
    net->Gs.push_back(g);
  }
  MCK(cudaMalloc(&net->X, rows * net->nin * sizeof(float)));
  MCK(cudaMalloc(&net->y, rows * sizeof(float)));
  MCK(cudaMalloc(&net->out, rows * sizeof(float)));
  MCK(cudaMalloc(&net->gout, rows * sizeof(float)));
  MCK(cudaMalloc(&net->partial, ((rows + 255) / 256) * sizeof(double)));
  net->cap = rows;
  return MW3_OK;
}

dim3 tgrid(int M, int N, int nsplit = 1) {
  return dim3((N + TBN - 1) / TBN, (M + TBM - 1) / TBM, nsplit);
}

// forward on rows already in net->X; output in net->out (Zs[L-1])
int forward(mw3_mlp* net, long n) {
  const int L = (int)net->sizes.size() - 1;
  const float* in = net->X;
  for (int l = 0; l < L; ++l) {
    const int K = net->sizes[l], N = net->sizes[l + 1];
    // A = activations [n][K] (FP32), B[k][o] = W[o][k] (BF16 weights, stored [o][k])
    const int mode = (l < L - 1) ? 0 : 1;
    float* C = (l < L - 1) ? net->Zs[l] : net->out;
    k_mlp_gemm_t<false, false, true, true><<<tgrid((int)n, N), 256>>>(
        (int)n, N, K, K, in, K, net->ph + net->woff[l], K, C, N, net->p + net->boff[l], nullptr,
        net->Hs[l], mode);
    in = net->Hs[l];
  }
  MCK(cudaGetLastError());
  return MW3_OK;
}

// backward from net->gout (dL/dout); gradients into net->g (flat)
int backward(mw3_mlp* net, long n) {
  const int L = (int)net->sizes.size() - 1;
  const float* g = net->gout;
  for (int l = L - 1; l >= 0; --l) {
    const int K = net->sizes[l], N = net->sizes[l + 1];
    const float* a_in = (l == 0) ? net->X : net->Hs[l - 1];
    // dW[o][i] = sum_r g[r][o] a_in[r][i]: M = N (o), N = K (i), K = n (r); A(o, r) = g[r][o]
    // (stored transposed), B(r, i) = a_in[r][i]; the batch is split into chunks of 512 rows
    // whose partial products are summed in chunk order
    {
      const int kchunk = 512;
      const int nsplit = (int)((n + kchunk - 1) / kchunk);
      const long need = (long)nsplit * N * K;
      if (need > net->split_cap) {
        cudaFree(net->split);
        MCK(cudaMalloc(&net->split, need * sizeof(float)));
        net->split_cap = need;
      }
      k_mlp_gemm_t<true, false, false, false><<<tgrid(N, K, nsplit), 256>>>(
          N, K, (int)n, kchunk, g, N, a_in, K, net->split, K, nullptr, nullptr, nullptr, 3);
      const long ne = (long)N * K;
      k_sum_splits<<<(unsigned)std::min<long>((ne + 255) / 256, 1024), 256>>>(
          net->split, nsplit, ne, net->g + net->woff[l]);
    }
    {
      const int nchunk = (int)((n + kColChunk - 1) / kColChunk);
      k_colsum_part<<<dim3((N + 31) / 32, nchunk), 256>>>(g, (int)n, N, net->split);
      k_sum_splits<<<(N + 255) / 256, 256>>>(net->split, nchunk, N, net->g + net->boff[l]);
    }
    if (l > 0) {
      // g_prev[r][i] = sum_o g[r][o] W[o][i] * gelu'(Z_(l-1)[r][i])
      // A(r, o) = g[r][o], B(o, i) = W[o][i] (BF16)
      k_mlp_gemm_t<false, false, false, true><<<tgrid((int)n, K), 256>>>(
          (int)n, K, N, N, g, N, net->ph + net->woff[l], K, net->Gs[l - 1], K, nullptr,
          net->Zs[l - 1], nullptr, 2);
      g = net->Gs[l - 1];
    }
  }
  MCK(cudaGetLastError());
  return MW3_OK;
}

double mse_and_grad(mw3_mlp* net, long n, const float* y) {
  const int nb = (int)((n + 255) / 256);
  k_mse<<<nb, 256>>>(net->out, y, (int)n, net->gout, net->partial);
  std::vector<double> h(nb);
  cudaMemcpy(h.data(), net->partial, nb * 8, cudaMemcpyDeviceToHost);
  double s = 0;
  for (double x : h) s += x;
  return s / (double)n;
}

uint16_t bf16_bits(float f) {  // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  return (uint16_t)(u >> 16);
}

int upload_params(mw3_mlp* net, const std::vector<float>& p) {
  std::vector<uint16_t> hb(p.size());
  for (size_t i = 0; i < p.size(); ++i) hb[i] = bf16_bits(p[i]);
  MCK(cudaMemcpy(net->p, p.data(), p.size() * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(net->ph, hb.data(), hb.size() * 2, cudaMemcpyHostToDevice));
  return MW3_OK;
}

}  // namespace

extern "C" {

int mw3_mlp_create(mw3_mlp** out, int device, int n_in, int width, int depth,
                   unsigned long long seed) {
  if (!out || n_in < 1 || width < 1 || depth < 1 || n_in > 64 || width > 4096 || depth > 16)
    return MW3_ERR_BAD_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return MW3_ERR_CUDA;
  mw3_mlp* net = new (std::nothrow) mw3_mlp();
  if (!net) return MW3_ERR_OOM;
  net->device = device;
  net->nin = n_in;
  net->width = width;
  net->depth = depth;
  net->sizes.push_back(n_in);
  for (int l = 0; l < depth; ++l) net->sizes.push_back(width);
  net->sizes.push_back(1);
  long off = 0;
  std::vector<unsigned char> mask;
  for (size_t l = 0; l + 1 < net->sizes.size(); ++l) {
    const long nw = (long)net->sizes[l] * net->sizes[l + 1];
    net->woff.push_back(off);
    off += nw;
    mask.insert(mask.end(), nw, 1);
    net->boff.push_back(off);
    off += net->sizes[l + 1];
    mask.insert(mask.end(), net->sizes[l + 1], 0);
  }
  net->nparam = off;
  const size_t n = (size_t)off;
  if (cudaMalloc(&net->p, n * 4) != cudaSuccess || cudaMalloc(&net->ph, n * 2) != cudaSuccess ||
      cudaMalloc(&net->g, n * 4) != cudaSuccess || cudaMalloc(&net->m, n * 4) != cudaSuccess ||
      cudaMalloc(&net->v, n * 4) != cudaSuccess || cudaMalloc(&net->wmask, n) != cudaSuccess) {
    delete net;
    return MW3_ERR_OOM;
  }
  cudaMemcpy(net->wmask, mask.data(), n, cudaMemcpyHostToDevice);
  cudaMemset(net->m, 0, n * 4);
  cudaMemset(net->v, 0, n * 4);
  // He-normal weights, zero biases (seeded, host generator)
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::vector<float> p(n, 0.f);
  for (size_t l = 0; l + 1 < net->sizes.size(); ++l) {
    const double sd = std::sqrt(2.0 / net->sizes[l]);
    const long nw = (long)net->sizes[l] * net->sizes[l + 1];
    for (long i = 0; i < nw; ++i) p[net->woff[l] + i] = (float)(nd(rng) * sd);
  }
  int st = upload_params(net, p);
  if (st) {
    delete net;
    return st;
  }
  *out = net;
  return MW3_OK;
}

void mw3_mlp_destroy(mw3_mlp* net) {
  if (!net) return;
  cudaSetDevice(net->device);
  free_acts(net);
  cudaFree(net->p);
  cudaFree(net->ph);
  cudaFree(net->g);
  cudaFree(net->m);
  cudaFree(net->v);
  cudaFree(net->wmask);
  cudaFree(net->Xall);
  cudaFree(net->yall);
  cudaFree(net->idx);
  cudaFree(net->split);
  delete net;
}

const char* mw3_mlp_last_error(const mw3_mlp* net) { return net ? net->err.c_str() : ""; }

long mw3_mlp_num_params(const mw3_mlp* net) { return net ? net->nparam : -1; }

int mw3_mlp_set_params(mw3_mlp* net, const double* flat) {
  if (!net || !flat) return MW3_ERR_BAD_ARG;
  cudaSetDevice(net->device);
  std::vector<float> p(flat, flat + net->nparam);
  net->step = 0;
  cudaMemset(net->m, 0, net->nparam * 4);
  cudaMemset(net->v, 0, net->nparam * 4);
  return upload_params(net, p);
}

int mw3_mlp_get_params(mw3_mlp* net, double* flat) {
  if (!net || !flat) return MW3_ERR_BAD_ARG;
  cudaSetDevice(net->device);
  std::vector<float> p(net->nparam);
  MCK(cudaMemcpy(p.data(), net->p, p.size() * 4, cudaMemcpyDeviceToHost));
  for (long i = 0; i < net->nparam; ++i) flat[i] = p[i];
  return MW3_OK;
}

int mw3_mlp_forward(mw3_mlp* net, const float* X, long n, float* y) {
  if (!net || !X || !y || n < 0) return MW3_ERR_BAD_ARG;
  cudaSetDevice(net->device);
  const long chunk = 65536;
  for (long r0 = 0; r0 < n; r0 += chunk) {
    const long rows = std::min(chunk, n - r0);
    int st = ensure_cap(net, rows);
    if (st) return st;
    MCK(cudaMemcpy(net->X, X + r0 * net->nin, rows * net->nin * 4, cudaMemcpyHostToDevice));
    if ((st = forward(net, rows))) return st;
    MCK(cudaMemcpy(y + r0, net->out, rows * 4, cudaMemcpyDeviceToHost));
  }
  return MW3_OK;
}

int mw3_mlp_loss_grad(mw3_mlp* net, const float* X, const float* y, long n, double* loss,
                      double* grad) {
  if (!net || !X || !y || n < 1) return MW3_ERR_BAD_ARG;
  cudaSetDevice(net->device);
  int st = ensure_cap(net, n);
  if (st) return st;
  MCK(cudaMemcpy(net->X, X, n * net->nin * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(net->y, y, n * 4, cudaMemcpyHostToDevice));
  if ((st = forward(net, n))) return st;
  const double l = mse_and_grad(net, n, net->y);
  if ((st = backward(net, n))) return st;
  if (loss) *loss = l;
  if (grad) {
    std::vector<float> g(net->nparam);
    MCK(cudaMemcpy(g.data(), net->g, g.size() * 4, cudaMemcpyDeviceToHost));
    for (long i = 0; i < net->nparam; ++i) grad[i] = g[i];
  }
  return MW3_OK;
}

int mw3_mlp_train(mw3_mlp* net, const float* X, const float* y, long n, int epochs, int batch,
                  double lr, double wd, unsigned long long seed, double* final_loss) {
  if (!net || !X || !y || n < 1 || epochs < 0 || batch < 1) return MW3_ERR_BAD_ARG;
  cudaSetDevice(net->device);
  if (n != net->nall) {
    cudaFree(net->Xall);
    cudaFree(net->yall);
    cudaFree(net->idx);
    MCK(cudaMalloc(&net->Xall, n * net->nin * 4));
    MCK(cudaMalloc(&net->yall, n * 4));
    MCK(cudaMalloc(&net->idx, n * 4));
    net->nall = n;
  }
  MCK(cudaMemcpy(net->Xall, X, n * net->nin * 4, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(net->yall, y, n * 4, cudaMemcpyHostToDevice));
  int st = ensure_cap(net, batch);
  if (st) return st;
  std::mt19937_64 rng(seed);
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  double last = 0;
  const float b1 = 0.9f, b2 = 0.999f;
  // per-step losses stay on the device until the end of the epoch, so the steps are queued
  // without a host round trip each
  const long steps_max = std::max<long>(1, n / batch + 1);
  double* dloss = nullptr;
  MCK(cudaMalloc(&dloss, steps_max * sizeof(double)));
  std::vector<double> hloss(steps_max);
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(perm.begin(), perm.end(), rng);
    MCK(cudaMemcpy(net->idx, perm.data(), n * 4, cudaMemcpyHostToDevice));
    long cnt = 0;
    for (long r0 = 0; r0 + batch <= n || (r0 == 0 && n < batch); r0 += batch) {
      const long rows = std::min<long>(batch, n - r0);
      k_gather<<<(int)((rows + 255) / 256), 256>>>(net->Xall, net->yall, net->idx + r0, (int)rows,
                                                    net->nin, net->X, net->y);
      if ((st = forward(net, rows))) {
        cudaFree(dloss);
        return st;
      }
      const int nb = (int)((rows + 255) / 256);
      k_mse<<<nb, 256>>>(net->out, net->y, (int)rows, net->gout, net->partial);
      k_loss_sum<<<1, 1>>>(net->partial, nb, (double)rows, dloss + cnt);
      if ((st = backward(net, rows))) {
        cudaFree(dloss);
        return st;
      }
      net->step += 1;
      const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
      k_adamw<<<(int)((net->nparam + 255) / 256), 256>>>(net->p, net->g, net->m, net->v, net->ph,
                                                         net->wmask, net->nparam, (float)lr, b1,
                                                         b2, 1e-8f, (float)wd, c1, c2);
      ++cnt;
      if (rows < batch) break;
    }
    if (cudaMemcpy(hloss.data(), dloss, cnt * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaFree(dloss);
      return mfail(net, MW3_ERR_CUDA, "mw3_mlp_train: loss read-back failed");
    }
    double sum = 0;
    for (long i = 0; i < cnt; ++i) sum += hloss[i];
    last = cnt ? sum / cnt : 0;
  }
  cudaFree(dloss);
  MCK(cudaDeviceSynchronize());
  if (final_loss) *final_loss = last;
  return MW3_OK;
}

}  // extern "C"
