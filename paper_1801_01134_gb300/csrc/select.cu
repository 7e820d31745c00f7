// Block-shape selection: features without conversion, a timing recorder,
// the paper-style polynomial predictor and a small MLP trained on the GPU.
//
// The paper picks a kernel before converting the matrix from the average
// number of values per block, Avg(r,c) = N_nnz / N_blocks(r,c), which is
// cheap to count (section "Performance prediction and optimal kernel
// selection"), through one fitted polynomial per kernel (section "Performance
// polynomial interpolation"); its conclusion asks for richer inputs. Here:
//   * features: N_blocks for all twelve shapes and the row-length sum, sum
//     of squares and maximum, counted from the CSR structure by the kernels
//     of counts.cu (runs between wide gaps for r = 1, one merge per interval
//     and r otherwise);
//   * spc5_time_formats: converts to each shape and times the SpMV (the
//     exhaustive choice, and the training targets);
//   * a least-squares polynomial per format (Householder QR on the
//     Vandermonde matrix of Avg(r,c));
//   * an MLP 16 -> 64 -> 64 -> 12 (ReLU, float32) scoring the formats, trained
//     with mean squared error and Adam by one fused kernel per minibatch step
//     (forward, loss gradient, backward, update inside one CTA, so the step is
//     deterministic); the layers are far too small for tensor cores to pay.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "internal.cuh"

namespace spc5 {
namespace {

constexpr int kNO = SPC5_NFORMATS;   // 12
constexpr int kH = 64;

// ----------------------------------------------------------------- MLP
// Parameter layout (float32, flat) for NF inputs: W1[64][NF], b1[64],
// W2[64][64], b2[64], W3[12][64], b3[12]. NF = 16 (the selection features)
// or 20 (the extended features: plus x-access locality, short rows and the
// SM fraction, see spc5_features_ext).
template <int NF>
struct Mlp {
  static constexpr int oW1 = 0, ob1 = oW1 + kH * NF, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
                       ob3 = oW3 + kNO * kH, NP = ob3 + kNO;
};
constexpr int kNF = SPC5_NFEATURES;  // 16
constexpr int kNP = Mlp<kNF>::NP;    // 6028 parameters
constexpr int kMaxBatch = 32;  // keeps the step's activations in static shared memory
constexpr int kStepThreads = 1024;

// One training step on a minibatch of B <= 32 samples (rows idx[0..B) of X and
// Y, with the 0/1 mask M saying which targets exist): forward, mean squared
// error gradient, backward, Adam update of the parameters, all in one CTA.
template <int NF>
__global__ void __launch_bounds__(kStepThreads) k_mlp_step(float* __restrict__ P, float* __restrict__ mom,
                                                           float* __restrict__ vel, const float* __restrict__ X,
                                                           const float* __restrict__ Y, const float* __restrict__ Mk,
                                                           const int32_t* __restrict__ idx, int B, int t, float lr,
                                                           float* __restrict__ loss_out, float* __restrict__ grad_out) {
  constexpr int oW1 = Mlp<NF>::oW1, ob1 = Mlp<NF>::ob1, oW2 = Mlp<NF>::oW2, ob2 = Mlp<NF>::ob2, oW3 = Mlp<NF>::oW3,
                ob3 = Mlp<NF>::ob3, kNP = Mlp<NF>::NP, kNF = NF;
  __shared__ float xs[kMaxBatch][kNF];
  __shared__ float z1[kMaxBatch][kH], z2[kMaxBatch][kH];  // pre-activations, then reused for gradients
  __shared__ float h1[kMaxBatch][kH], h2[kMaxBatch][kH];
  __shared__ float dout[kMaxBatch][kNO];
  __shared__ float red[kStepThreads / 32];
  const int tid = threadIdx.x;
  for (int e = tid; e < B * kNF; e += kStepThreads) xs[e / kNF][e % kNF] = X[(int64_t)idx[e / kNF] * kNF + e % kNF];
  __syncthreads();
  // layer 1
  for (int e = tid; e < B * kH; e += kStepThreads) {
    const int s = e / kH, j = e % kH;
    float a = P[ob1 + j];
    for (int q = 0; q < kNF; ++q) a = fmaf(P[oW1 + j * kNF + q], xs[s][q], a);
    z1[s][j] = a;
    h1[s][j] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < B * kH; e += kStepThreads) {
    const int s = e / kH, j = e % kH;
    float a = P[ob2 + j];
    for (int q = 0; q < kH; ++q) a = fmaf(P[oW2 + j * kH + q], h1[s][q], a);
    z2[s][j] = a;
    h2[s][j] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  // outputs, masked squared error and its gradient
  float msum = 0.f;
  for (int s = 0; s < B; ++s)
    for (int o = 0; o < kNO; ++o) msum += Mk[(int64_t)idx[s] * kNO + o];  // every thread: same value
  float lsum = 0.f;
  for (int e = tid; e < B * kNO; e += kStepThreads) {
    const int s = e / kNO, o = e % kNO;
    float a = P[ob3 + o];
    for (int q = 0; q < kH; ++q) a = fmaf(P[oW3 + o * kH + q], h2[s][q], a);
    const float m = Mk[(int64_t)idx[s] * kNO + o];
    const float d = a - Y[(int64_t)idx[s] * kNO + o];
    dout[s][o] = msum > 0.f ? 2.f * m * d / msum : 0.f;
    lsum += m * d * d;
  }
  // loss (block sum, fixed order)
  for (int d = 16; d >= 1; d >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, d);
  if ((tid & 31) == 0) red[tid >> 5] = lsum;
  __syncthreads();
  if (tid == 0) {
    float l = 0.f;
    for (int k = 0; k < kStepThreads / 32; ++k) l += red[k];
    if (loss_out) *loss_out = msum > 0.f ? l / msum : 0.f;
  }
  // dH2 -> dZ2 (into z2)
  for (int e = tid; e < B * kH; e += kStepThreads) {
    const int s = e / kH, j = e % kH;
    float a = 0.f;
    for (int o = 0; o < kNO; ++o) a = fmaf(dout[s][o], P[oW3 + o * kH + j], a);
    z2[s][j] = z2[s][j] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // dH1 -> dZ1 (into z1)
  for (int e = tid; e < B * kH; e += kStepThreads) {
    const int s = e / kH, j = e % kH;
    float a = 0.f;
    for (int o = 0; o < kH; ++o) a = fmaf(z2[s][o], P[oW2 + o * kH + j], a);
    z1[s][j] = z1[s][j] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // gradients (sum over the batch in sample order) and the Adam update; each
  // parameter is owned by one thread
  const float b1c = 1.f - powf(0.9f, (float)t), b2c = 1.f - powf(0.999f, (float)t);
  for (int p = tid; p < kNP; p += kStepThreads) {
    float g = 0.f;
    if (p < ob1) {
      const int j = (p - oW1) / kNF, q = (p - oW1) % kNF;
      for (int s = 0; s < B; ++s) g = fmaf(z1[s][j], xs[s][q], g);
    } else if (p < oW2) {
      const int j = p - ob1;
      for (int s = 0; s < B; ++s) g += z1[s][j];
    } else if (p < ob2) {
      const int j = (p - oW2) / kH, q = (p - oW2) % kH;
      for (int s = 0; s < B; ++s) g = fmaf(z2[s][j], h1[s][q], g);
    } else if (p < oW3) {
      const int j = p - ob2;
      for (int s = 0; s < B; ++s) g += z2[s][j];
    } else if (p < ob3) {
      const int o = (p - oW3) / kH, q = (p - oW3) % kH;
      for (int s = 0; s < B; ++s) g = fmaf(dout[s][o], h2[s][q], g);
    } else {
      const int o = p - ob3;
      for (int s = 0; s < B; ++s) g += dout[s][o];
    }
    if (grad_out) grad_out[p] = g;
    if (lr > 0.f) {
      const float m = 0.9f * mom[p] + 0.1f * g;
      const float v = 0.999f * vel[p] + 0.001f * g * g;
      mom[p] = m;
      vel[p] = v;
      P[p] -= lr * (m / b1c) / (sqrtf(v / b2c) + 1e-8f);
    }
  }
}

// scores of N samples: one thread per (sample, output); hidden layers of a
// sample recomputed per output is wasteful but N is small; instead one thread
// per sample with the activations in local arrays
template <int NF>
__global__ void __launch_bounds__(128) k_mlp_infer(const float* __restrict__ P, const float* __restrict__ X, int N,
                                                   float* __restrict__ out) {
  constexpr int oW1 = Mlp<NF>::oW1, ob1 = Mlp<NF>::ob1, oW2 = Mlp<NF>::oW2, ob2 = Mlp<NF>::ob2, oW3 = Mlp<NF>::oW3,
                ob3 = Mlp<NF>::ob3, kNF = NF;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  float a1[kH], a2[kH];
  for (int j = 0; j < kH; ++j) {
    float a = P[ob1 + j];
    for (int q = 0; q < kNF; ++q) a = fmaf(P[oW1 + j * kNF + q], X[(int64_t)s * kNF + q], a);
    a1[j] = a > 0.f ? a : 0.f;
  }
  for (int j = 0; j < kH; ++j) {
    float a = P[ob2 + j];
    for (int q = 0; q < kH; ++q) a = fmaf(P[oW2 + j * kH + q], a1[q], a);
    a2[j] = a > 0.f ? a : 0.f;
  }
  for (int o = 0; o < kNO; ++o) {
    float a = P[ob3 + o];
    for (int q = 0; q < kH; ++q) a = fmaf(P[oW3 + o * kH + q], a2[q], a);
    out[(int64_t)s * kNO + o] = a;
  }
}

struct DBuf {
  void* p = nullptr;
  ~DBuf() {
    if (p) cudaFree(p);
  }
};

// Householder QR least squares: minimise ||V c - y|| for V (N x k), N >= k.
bool lstsq(std::vector<double> V, std::vector<double> y, int N, int k, double* c) {
  for (int j = 0; j < k; ++j) {
    double nrm = 0;
    for (int i = j; i < N; ++i) nrm += V[(size_t)i * k + j] * V[(size_t)i * k + j];
    nrm = std::sqrt(nrm);
    if (nrm == 0) return false;
    const double alpha = V[(size_t)j * k + j] > 0 ? -nrm : nrm;
    std::vector<double> v((size_t)N, 0.0);
    for (int i = j; i < N; ++i) v[(size_t)i] = V[(size_t)i * k + j];
    v[(size_t)j] -= alpha;
    double vv = 0;
    for (int i = j; i < N; ++i) vv += v[(size_t)i] * v[(size_t)i];
    if (vv == 0) continue;
    for (int col = j; col < k; ++col) {
      double d = 0;
      for (int i = j; i < N; ++i) d += v[(size_t)i] * V[(size_t)i * k + col];
      d = 2 * d / vv;
      for (int i = j; i < N; ++i) V[(size_t)i * k + col] -= d * v[(size_t)i];
    }
    double d = 0;
    for (int i = j; i < N; ++i) d += v[(size_t)i] * y[(size_t)i];
    d = 2 * d / vv;
    for (int i = j; i < N; ++i) y[(size_t)i] -= d * v[(size_t)i];
  }
  for (int j = k - 1; j >= 0; --j) {
    double s = y[(size_t)j];
    for (int q = j + 1; q < k; ++q) s -= V[(size_t)j * k + q] * c[q];
    if (V[(size_t)j * k + j] == 0) return false;
    c[j] = s / V[(size_t)j * k + j];
  }
  return true;
}

}  // namespace

spc5_status features_impl(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx, double* f,
                          cudaStream_t s) {
  DBuf acc;
  cudaError_t e = cudaMalloc(&acc.p, sizeof(unsigned long long) * 16);
  if (e == cudaSuccess) e = launch_block_counts(n, nnz, rowptr, colidx, (unsigned long long*)acc.p, s);
  unsigned long long h[15];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "features");
  for (int q = 0; q < 12; ++q) f[q] = h[q] ? (double)nnz / (double)h[q] : 0.0;
  const double mean = n > 0 ? (double)h[12] / (double)n : 0.0;
  const double var = n > 0 ? (double)h[13] / (double)n - mean * mean : 0.0;
  f[12] = mean;
  f[13] = var > 0 ? std::sqrt(var) : 0.0;
  f[14] = (double)h[14];
  f[15] = std::log10((double)(n > 1 ? n : 1));
  return SPC5_OK;
}

// Matrix statistics beyond Avg(r,c) for the extended features: the summed
// distance |col - row| of the entries from the diagonal (how far the x
// gathers of a row stray from it; the paper names the block distribution's
// effect on the x accesses as what Avg alone cannot tell) and the number of
// rows of at most two entries. A warp per 32 rows, its lanes splitting each
// row's entries; integer sums, so the result does not depend on the order.
__global__ void k_matrix_stats(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                               unsigned long long* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const int64_t r0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
  if (r0 >= n) return;  // whole warp
  unsigned long long dist = 0, shortrows = 0;
  const int64_t r1 = r0 + 32 < n ? r0 + 32 : n;
  for (int64_t i = r0; i < r1; ++i) {
    const int64_t a = rowptr[i], b = rowptr[i + 1];
    if (lane == 0 && b - a <= 2) ++shortrows;
    for (int64_t p = a + lane; p < b; p += 32) {
      const int64_t d = (int64_t)colidx[p] - i;
      dist += (unsigned long long)(d < 0 ? -d : d);
    }
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) dist += __shfl_xor_sync(0xffffffffu, dist, d);
  if (lane == 0) {
    atomicAdd(acc, dist);
    atomicAdd(acc + 1, shortrows);
  }
}

spc5_status features_ext_impl(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                              double sm_frac, double* f, cudaStream_t s) {
  spc5_status st = features_impl(n, nnz, rowptr, colidx, f, s);
  if (st != SPC5_OK) return st;
  DBuf acc;
  cudaError_t e = cudaMalloc(&acc.p, sizeof(unsigned long long) * 2);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long) * 2, s);
  if (e == cudaSuccess && n > 0) {
    const int64_t warps = (n + 31) / 32;
    k_matrix_stats<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(n, rowptr, colidx,
                                                                       (unsigned long long*)acc.p);
    e = cudaGetLastError();
  }
  unsigned long long h[2] = {0ull, 0ull};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "features_ext");
  const double mean_dist = nnz > 0 ? (double)h[0] / (double)nnz : 0.0;
  f[16] = n > 0 ? mean_dist / (double)n : 0.0;
  f[17] = std::log10(1.0 + mean_dist);
  f[18] = n > 0 ? (double)h[1] / (double)n : 0.0;
  f[19] = sm_frac;
  return SPC5_OK;
}

spc5_status mlp_train_impl(float* P, const float* X, const float* Y, const float* M, int N, int epochs, int batch,
                           float lr, uint64_t seed, float* loss_hist, cudaStream_t s, int nfeat) {
  if (batch < 1 || batch > kMaxBatch) return fail(SPC5_EINVAL, "mlp_train: batch must be in [1, 32]");
  if (nfeat != 16 && nfeat != 20) return fail(SPC5_EINVAL, "mlp_train: nfeat must be 16 or 20");
  const int kNP = mlp_param_count(nfeat);
  const int steps_per_epoch = (N + batch - 1) / batch;
  DBuf mom, vel, idx, loss;
  cudaError_t e = cudaMalloc(&mom.p, sizeof(float) * kNP);
  if (e == cudaSuccess) e = cudaMalloc(&vel.p, sizeof(float) * kNP);
  if (e == cudaSuccess) e = cudaMalloc(&idx.p, sizeof(int32_t) * (size_t)N);
  if (e == cudaSuccess) e = cudaMalloc(&loss.p, sizeof(float) * (size_t)steps_per_epoch);
  if (e == cudaSuccess) e = cudaMemsetAsync(mom.p, 0, sizeof(float) * kNP, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(vel.p, 0, sizeof(float) * kNP, s);
  if (e != cudaSuccess) return cuda_fail(e, "mlp_train: workspace");
  std::mt19937_64 rng(seed);
  std::vector<int32_t> order((size_t)N);
  std::vector<float> lh((size_t)steps_per_epoch);
  int t = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = 0; i < N; ++i) order[(size_t)i] = i;
    std::shuffle(order.begin(), order.end(), rng);
    e = cudaMemcpyAsync(idx.p, order.data(), sizeof(int32_t) * (size_t)N, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "mlp_train: indices");
    for (int st = 0; st < steps_per_epoch; ++st) {
      const int b0 = st * batch;
      const int B = N - b0 < batch ? N - b0 : batch;
      ++t;
      if (nfeat == 16)
        k_mlp_step<16><<<1, kStepThreads, 0, s>>>(P, (float*)mom.p, (float*)vel.p, X, Y, M, (const int32_t*)idx.p + b0,
                                                  B, t, lr, (float*)loss.p + st, nullptr);
      else
        k_mlp_step<20><<<1, kStepThreads, 0, s>>>(P, (float*)mom.p, (float*)vel.p, X, Y, M, (const int32_t*)idx.p + b0,
                                                  B, t, lr, (float*)loss.p + st, nullptr);
    }
    e = cudaMemcpyAsync(lh.data(), loss.p, sizeof(float) * (size_t)steps_per_epoch, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "mlp_train: step");
    if (loss_hist) {
      double a = 0;
      for (int st = 0; st < steps_per_epoch; ++st) a += lh[(size_t)st];
      loss_hist[ep] = (float)(a / steps_per_epoch);
    }
  }
  return SPC5_OK;
}

spc5_status mlp_grad_impl(const float* P, const float* X, const float* Y, const float* M, int B, float* loss,
                          float* grad, cudaStream_t s, int nfeat) {
  if (B < 1 || B > kMaxBatch) return fail(SPC5_EINVAL, "mlp_grad: batch must be in [1, 32]");
  if (nfeat != 16 && nfeat != 20) return fail(SPC5_EINVAL, "mlp_grad: nfeat must be 16 or 20");
  const int kNP = mlp_param_count(nfeat);
  std::vector<int32_t> order((size_t)B);
  for (int i = 0; i < B; ++i) order[(size_t)i] = i;
  DBuf idx, l, Pc;
  cudaError_t e = cudaMalloc(&idx.p, sizeof(int32_t) * (size_t)B);
  if (e == cudaSuccess) e = cudaMalloc(&l.p, sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&Pc.p, sizeof(float) * kNP);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Pc.p, P, sizeof(float) * kNP, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(idx.p, order.data(), sizeof(int32_t) * (size_t)B, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "mlp_grad: workspace");
  // lr = 0: gradient only, the parameter copy is left as it is
  if (nfeat == 16)
    k_mlp_step<16><<<1, kStepThreads, 0, s>>>((float*)Pc.p, nullptr, nullptr, X, Y, M, (const int32_t*)idx.p, B, 1,
                                              0.f, (float*)l.p, grad);
  else
    k_mlp_step<20><<<1, kStepThreads, 0, s>>>((float*)Pc.p, nullptr, nullptr, X, Y, M, (const int32_t*)idx.p, B, 1,
                                              0.f, (float*)l.p, grad);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(loss, l.p, sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "mlp_grad");
  return SPC5_OK;
}

spc5_status mlp_infer_impl(const float* P, const float* X, int N, float* out, cudaStream_t s, int nfeat) {
  if (nfeat != 16 && nfeat != 20) return fail(SPC5_EINVAL, "mlp_infer: nfeat must be 16 or 20");
  if (N > 0 && nfeat == 16) k_mlp_infer<16><<<(unsigned)((N + 127) / 128), 128, 0, s>>>(P, X, N, out);
  if (N > 0 && nfeat == 20) k_mlp_infer<20><<<(unsigned)((N + 127) / 128), 128, 0, s>>>(P, X, N, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mlp_infer");
  return SPC5_OK;
}

spc5_status poly_fit_impl(const double* avg, const double* perf, int N, int degree, double* coef) {
  const int k = degree + 1;
  if (degree < 0 || degree > 6 || N < k) return fail(SPC5_EINVAL, "poly_fit: need 0 <= degree <= 6 and N > degree");
  for (int f = 0; f < kNO; ++f) {
    std::vector<double> V((size_t)N * k), y((size_t)N);
    for (int i = 0; i < N; ++i) {
      double p = 1.0;
      for (int j = 0; j < k; ++j) {
        V[(size_t)i * k + j] = p;
        p *= avg[(size_t)i * kNO + f];
      }
      y[(size_t)i] = perf[(size_t)i * kNO + f];
    }
    if (!lstsq(V, y, N, k, coef + (size_t)f * k)) return fail(SPC5_EINVAL, "poly_fit: rank-deficient data");
  }
  return SPC5_OK;
}

int poly_select_impl(const double* coef, int degree, const double* feat, double* est) {
  int best = 0;
  for (int f = 0; f < kNO; ++f) {
    double v = 0.0;
    for (int j = degree; j >= 0; --j) v = v * feat[f] + coef[(size_t)f * (degree + 1) + j];
    est[f] = v;
    if (v > est[best]) best = f;
  }
  return best;
}

// The paper's parallel predictor: per format, a least-squares polynomial of
// the performance in two variables, Avg(r,c) and the amount of parallel
// hardware (threads there, the fraction of the SMs here): every monomial
// Avg^a s^b with a + b <= degree, ordered by total degree t = a + b, then by b.
int poly2_terms(int degree) { return (degree + 1) * (degree + 2) / 2; }

static void poly2_row(double avg, double s, int degree, double* row) {
  int q = 0;
  for (int t = 0; t <= degree; ++t)
    for (int b = 0; b <= t; ++b) {
      const int a = t - b;
      double v = 1.0;
      for (int k = 0; k < a; ++k) v *= avg;
      for (int k = 0; k < b; ++k) v *= s;
      row[q++] = v;
    }
}

spc5_status poly2_fit_impl(const double* avg, const double* sfrac, const double* perf, int N, int degree,
                           double* coef) {
  if (degree < 0 || degree > 4) return fail(SPC5_EINVAL, "poly2_fit: need 0 <= degree <= 4");
  const int k = poly2_terms(degree);
  if (N < k) return fail(SPC5_EINVAL, "poly2_fit: fewer samples than terms");
  for (int f = 0; f < kNO; ++f) {
    std::vector<double> V((size_t)N * k), y((size_t)N);
    for (int i = 0; i < N; ++i) {
      poly2_row(avg[(size_t)i * kNO + f], sfrac[i], degree, &V[(size_t)i * k]);
      y[(size_t)i] = perf[(size_t)i * kNO + f];
    }
    if (!lstsq(V, y, N, k, coef + (size_t)f * k)) return fail(SPC5_EINVAL, "poly2_fit: rank-deficient data");
  }
  return SPC5_OK;
}

int poly2_select_impl(const double* coef, int degree, const double* feat, double sfrac, double* est) {
  const int k = poly2_terms(degree);
  std::vector<double> row((size_t)k);
  int best = 0;
  for (int f = 0; f < kNO; ++f) {
    poly2_row(feat[f], sfrac, degree, row.data());
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += coef[(size_t)f * k + j] * row[(size_t)j];
    est[f] = v;
    if (v > est[best]) best = f;
  }
  return best;
}

int mlp_param_count(int nfeat) { return nfeat == 20 ? Mlp<20>::NP : Mlp<16>::NP; }

}  // namespace spc5
