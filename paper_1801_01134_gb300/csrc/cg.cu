// Conjugate gradients over beta(r,c) SpMV, in float64 and as mixed-precision
// iterative refinement (float64 residual / update / norms, float32 or bfloat16
// matrix with float32 vectors inside).
//
// The paper motivates fast SpMV by iterative solvers such as CG, which apply
// one matrix many times (Introduction). CG is Hestenes & Stiefel's; the
// refinement loop is the classical one (Wilkinson; Moler 1967):
//     r = b - A x (float64);  solve A d ~= r / ||r|| in float32;  x += ||r|| d.
// A third mode keeps one float32 CG recurrence and replaces its residual by the
// float64 one from time to time (reliable updates, Sleijpen & van der Vorst
// 1996), which needs about the float64 iteration count instead of paying for
// restarts.
// On GB300 float64 arithmetic is issue-bound (one float64 FMA warp-instruction
// per ~16 SM cycles), so moving the bulk of the work to float32 pays twice:
// half the bytes per SpMV and no float64 pipe in the inner loop.
//
// The iteration is ordered so that it takes two kernels. With beta from the
// previous iteration (0 at the start, p = q = 0):
//     q = A r + beta q,  p = r + beta p,  alpha = rho / (p.q)     (kernel 1)
//     x += alpha p,  r -= alpha q,  rho' = r.r,  beta = rho'/rho  (kernel 2)
// which is Hestenes-Stiefel CG with A p_k formed as A r_k + beta A p_{k-1}
// (equal in exact arithmetic), so the SpMV reads r and the p update rides in
// its epilogue instead of a third pass.
// Scalars (rho, p.q, alpha, beta) never leave the device inside an iteration:
// dot products reduce to per-block partials that the last block to finish
// sums in a fixed order (so results repeat run to run), writing the derived
// scalar too. The iteration can be captured once into a CUDA graph and
// replayed. The host reads the residual norm every `check_every` iterations.
#include <cmath>
#include <vector>

#include "spmv_beta.cuh"

namespace spc5 {
namespace {

constexpr int kThreads = 256;
// Grid caps (beyond them, warps stride over the work). Every block adds one
// same-address atomic to the reduction ticket, and those serialise at about
// 2.5 ns each on GB300, so a smaller grid finishes the reduction sooner:
// measured best at 4 blocks per SM for the fused SpMV, 2 for the vector
// updates (7-point Poisson 96^3, float64 CG 21.7 -> 17.4 ms).
constexpr int kSpmvBlocksPerSm = 4;
constexpr int kVecBlocksPerSm = 2;
enum { S_RHO = 0, S_PQ, S_ALPHA, S_BETA, S_RHONEW, S_NORM, S_COUNT = 8 };
// k_dot_final mode: the recurred residual was replaced (reliable update);
// beta = rho_new / rho_previous = s * beta / rho, then rho = s
constexpr int S_REPLACED = 100;
constexpr double kReliableDelta = 0.1;  // update when the recurred norm fell by this factor

template <class A>
__device__ __forceinline__ A block_sum(A v) {
  __shared__ A ws[kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  if (lane == 0) ws[w] = v;
  __syncthreads();
  A t = threadIdx.x < kThreads / 32 ? ws[threadIdx.x] : A(0);
  if (w == 0) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// part[block] = sum_i a[i] b[i] (grid-stride, accumulation type A)
template <class T, class A>
__global__ void __launch_bounds__(kThreads) k_dot_part(const T* __restrict__ a, const T* __restrict__ b, int64_t n,
                                                       A* __restrict__ part) {
  A s = 0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    s = fma((A)a[i], (A)b[i], s);
  s = block_sum<A>(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// One thread-block sums the partials in float64 in a fixed order and writes
// the scalar `what`, with its derived scalar:
//   S_PQ     -> alpha = rho / pq      (0 when pq == 0)
//   S_RHONEW -> beta = rhonew / rho, then rho = rhonew
//   S_RHO / S_NORM -> plain sum
template <class A>
__global__ void __launch_bounds__(kThreads) k_dot_final(const A* __restrict__ part, int nb, double* __restrict__ scal,
                                                        int what) {
  double s = 0;
  for (int i = threadIdx.x; i < nb; i += kThreads) s += (double)part[i];
  s = block_sum<double>(s);
  if (threadIdx.x == 0) {
    if (what == S_PQ) {
      scal[S_PQ] = s;
      scal[S_ALPHA] = s != 0.0 ? scal[S_RHO] / s : 0.0;
    } else if (what == S_RHONEW) {
      scal[S_RHONEW] = s;
      scal[S_BETA] = scal[S_RHO] != 0.0 ? s / scal[S_RHO] : 0.0;
      scal[S_RHO] = s;
    } else if (what == S_REPLACED) {
      scal[S_BETA] = scal[S_RHO] != 0.0 ? s * scal[S_BETA] / scal[S_RHO] : 0.0;
      scal[S_RHO] = s;
    } else {
      scal[what] = s;
    }
  }
}

// r = b - t (float64) and its partial r.r
__global__ void __launch_bounds__(kThreads) k_residual(double* __restrict__ r, const double* __restrict__ b,
                                                       const double* __restrict__ t, int64_t n,
                                                       double* __restrict__ part) {
  double s = 0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const double ri = b[i] - t[i];
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  s = block_sum<double>(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// start of an inner solve: r32 = r64 / ||r64||, p32 = q32 = x32 = 0, beta = 0
__global__ void __launch_bounds__(kThreads) k_inner_start(const double* __restrict__ r64, float* __restrict__ r32,
                                                          float* __restrict__ p32, float* __restrict__ q32,
                                                          float* __restrict__ x32, int64_t n, double* __restrict__ scal) {
  const double inv = scal[S_NORM] > 0.0 ? 1.0 / sqrt(scal[S_NORM]) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    r32[i] = (float)(r64[i] * inv);
    p32[i] = 0.0f;
    q32[i] = 0.0f;
    x32[i] = 0.0f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[S_BETA] = 0.0;
}

// x64 += ||r|| * x32
__global__ void __launch_bounds__(kThreads) k_inner_apply(double* __restrict__ x64, const float* __restrict__ x32,
                                                          int64_t n, const double* __restrict__ scal) {
  const double nr = sqrt(scal[S_NORM]);
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    x64[i] = fma(nr, (double)x32[i], x64[i]);
}

// reliable update: x64 += x32, x32 = 0
__global__ void __launch_bounds__(kThreads) k_fold_x(double* __restrict__ x64, float* __restrict__ x32, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    x64[i] += (double)x32[i];
    x32[i] = 0.0f;
  }
}

// r32 = (float) r64
__global__ void __launch_bounds__(kThreads) k_narrow(const double* __restrict__ r64, float* __restrict__ r32,
                                                     int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    r32[i] = (float)r64[i];
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_copy_vec(T* __restrict__ d, const T* __restrict__ s, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) d[i] = s[i];
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_zero_vec(T* __restrict__ d, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) d[i] = T(0);
}

// Last-block-done finish of a grid reduction: every block has stored its
// partial in part[blockIdx.x]; the block that arrives last (atomic ticket)
// sums all partials in index order - the same order on every run - and
// resets the ticket for the next kernel. Returns the total in that block
// (thread 0), and whether this block is the last one.
template <class A>
__device__ __forceinline__ bool finish_last_block(A* part, A mine, unsigned* ticket, double* total) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = mine;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  double s = 0;
  for (unsigned j = threadIdx.x; j < gridDim.x; j += kThreads) s += (double)__ldcg(part + j);
  s = block_sum<double>(s);
  if (threadIdx.x == 0) {
    *total = s;
    *ticket = 0u;
  }
  return true;
}

// q = A r + beta q and p = r + beta p over the short intervals, one lane per
// row (the SpMV kernel's row sum applied to r), fused with p.q; the last
// block writes scal[PQ] and scal[ALPHA].
template <int R, int C, class T, int U, int DEC>
__global__ void __launch_bounds__(kThreads) k_cg_spmv_dot(int64_t n, int64_t I, const int32_t* __restrict__ brp,
                                                          const int32_t* __restrict__ bcol,
                                                          const uint8_t* __restrict__ bmask,
                                                          const typename T::V* __restrict__ val,
                                                          const int64_t* __restrict__ valptr,
                                                          const typename T::X* __restrict__ r,
                                                          typename T::X* __restrict__ p, typename T::X* __restrict__ q,
                                                          typename T::A* part, unsigned* ticket,
                                                          double* __restrict__ scal) {
  using A = typename T::A;
  using X = typename T::X;
  constexpr int S = kWarp / R;
  const int lane = threadIdx.x & 31;
  const int i = lane % R;
  const X beta = (X)scal[S_BETA];
  const int64_t nwarps = (int64_t)gridDim.x * (kThreads / kWarp);
  const int64_t ntasks = (I + S - 1) / S;
  A prod = 0;
  // warps stride over the tasks (32/r intervals each) when the grid is capped
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntasks; task += nwarps) {
    const int64_t it = task * S + lane / R;
    if (it < I) {
      const int32_t b = __ldg(brp + it), bend = __ldg(brp + it + 1);
      const A acc = row_sum<R, C, T, U, DEC>(i, b, bend, val + __ldg(valptr + it), bcol, bmask, r);
      const int64_t row = it * R + i;
      if (row < n) {
        const X qn = fma(beta, q[row], (X)acc);
        const X pn = fma(beta, p[row], r[row]);
        q[row] = qn;
        p[row] = pn;
        prod = fma((A)pn, (A)qn, prod);
      }
    }
  }
  prod = block_sum<A>(prod);
  double tot;
  if (finish_last_block<A>(part, prod, ticket, &tot) && threadIdx.x == 0) {
    scal[S_PQ] = tot;
    scal[S_ALPHA] = tot != 0.0 ? scal[S_RHO] / tot : 0.0;
  }
}

// 16-byte vector of T (float4 / double2) for the streaming kernels
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int N = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int N = 2;
};

template <class T>
__device__ __forceinline__ T& lane_of(typename Vec16<T>::type& v, int k) {
  return reinterpret_cast<T*>(&v)[k];
}

// Non-fused epilogue (matrices with long intervals): w = A r came from the
// SpMV; q = w + beta q, p = r + beta p, p.q finished by the last block.
template <class T, class A>
__global__ void __launch_bounds__(kThreads) k_cg_pq(T* __restrict__ p, T* __restrict__ q, const T* __restrict__ r,
                                                    const T* __restrict__ w, int64_t n, double* __restrict__ scal,
                                                    A* part, unsigned* ticket) {
  const T beta = (T)scal[S_BETA];
  A prod = 0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const T qn = fma(beta, q[i], w[i]);
    const T pn = fma(beta, p[i], r[i]);
    q[i] = qn;
    p[i] = pn;
    prod = fma((A)pn, (A)qn, prod);
  }
  prod = block_sum<A>(prod);
  double tot;
  if (finish_last_block<A>(part, prod, ticket, &tot) && threadIdx.x == 0) {
    scal[S_PQ] = tot;
    scal[S_ALPHA] = tot != 0.0 ? scal[S_RHO] / tot : 0.0;
  }
}

// x += alpha p; r -= alpha q; r.r finished by the last block, which writes
// rhonew, beta = rhonew / rho and rho = rhonew. 16-byte loads and stores;
// element i's arithmetic is the same whichever thread does it.
template <class T, class A>
__global__ void __launch_bounds__(kThreads) k_cg_xr_fused(T* __restrict__ x, T* __restrict__ r,
                                                          const T* __restrict__ p, const T* __restrict__ q, int64_t n,
                                                          double* __restrict__ scal, A* part, unsigned* ticket) {
  using V = typename Vec16<T>::type;
  constexpr int N = Vec16<T>::N;
  const T alpha = (T)scal[S_ALPHA];
  A s = 0;
  const bool aligned = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(r) |
                         reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q)) & 15u) == 0;
  const int64_t nv = aligned ? n / N : 0;  // a caller's x may start anywhere: then all scalar
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t v = (int64_t)blockIdx.x * kThreads + threadIdx.x; v < nv; v += stride) {
    V xv = reinterpret_cast<const V*>(x)[v], rv = reinterpret_cast<const V*>(r)[v];
    const V pv = reinterpret_cast<const V*>(p)[v], qv = reinterpret_cast<const V*>(q)[v];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      lane_of<T>(xv, k) = fma(alpha, lane_of<T>(const_cast<V&>(pv), k), lane_of<T>(xv, k));
      const T ri = fma(-alpha, lane_of<T>(const_cast<V&>(qv), k), lane_of<T>(rv, k));
      lane_of<T>(rv, k) = ri;
      s = fma((A)ri, (A)ri, s);
    }
    reinterpret_cast<V*>(x)[v] = xv;
    reinterpret_cast<V*>(r)[v] = rv;
  }
  for (int64_t i = nv * N + (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
    x[i] = fma(alpha, p[i], x[i]);
    const T ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    s = fma((A)ri, (A)ri, s);
  }
  s = block_sum<A>(s);
  double tot;
  if (finish_last_block<A>(part, s, ticket, &tot) && threadIdx.x == 0) {
    scal[S_RHONEW] = tot;
    scal[S_BETA] = scal[S_RHO] != 0.0 ? tot / scal[S_RHO] : 0.0;
    scal[S_RHO] = tot;
  }
}

template <class T>
cudaError_t launch_fused_spmv_dot(const spc5_matrix* M, const void* r, void* p, void* q, void* part, unsigned* ticket,
                                  double* scal, cudaStream_t s) {
  using V = typename T::V;
  using X = typename T::X;
  using A = typename T::A;
#define SPC5_CASE(RR, CC)                                                                                         \
  if (M->r == RR && M->c == CC) {                                                                                 \
    constexpr int S = kWarp / RR;                                                                                 \
    const int64_t warps = (M->I + S - 1) / S;                                                                     \
    int64_t blocks = (warps * kWarp + kThreads - 1) / kThreads;                                                   \
    if (blocks > (int64_t)sm_count() * kSpmvBlocksPerSm) blocks = (int64_t)sm_count() * kSpmvBlocksPerSm;         \
    const unsigned grid = (unsigned)blocks;                                                                        \
    auto go = [&](auto kern) {                                                                                    \
      kern<<<grid, kThreads, 0, s>>>(M->n, M->I, M->block_rowptr, M->block_colidx, M->block_masks,               \
                                     (const V*)M->values, M->valptr, (const X*)r, (X*)p, (X*)q, (A*)part, ticket,  \
                                     scal);                                                                        \
    };                                                                                                            \
    if (M->variant == 16)                                                                                         \
      go(k_cg_spmv_dot<RR, CC, T, 1, 2>);                                                                         \
    else if (M->variant == 18)                                                                                    \
      go(k_cg_spmv_dot<RR, CC, T, 1, 3>);                                                                         \
    else                                                                                                          \
      go(k_cg_spmv_dot<RR, CC, T, 2, 0>);                                                                         \
    return cudaGetLastError();                                                                                    \
  }
  SPC5_CASE(1, 4) SPC5_CASE(1, 8) SPC5_CASE(1, 16)
  SPC5_CASE(2, 4) SPC5_CASE(2, 8) SPC5_CASE(2, 16)
  SPC5_CASE(4, 4) SPC5_CASE(4, 8) SPC5_CASE(4, 16)
  SPC5_CASE(8, 4) SPC5_CASE(8, 8) SPC5_CASE(8, 16)
#undef SPC5_CASE
  return cudaErrorInvalidValue;
}

struct Buf {
  void* p = nullptr;
  ~Buf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes > 0 ? bytes : 16); }
};

cudaError_t spmv_any(const spc5_matrix* h, const void* x, void* y, cudaStream_t s) {
  switch (h->vt) {
    case SPC5_F64: return launch_spmv_f64(h, x, y, false, s);
    case SPC5_F32: return launch_spmv_f32(h, x, y, false, s);
    default: return launch_spmv_bf16(h, x, y, false, s);
  }
}

// One CG iteration on the stream (vector type T, accumulation type A), in
// the order of the file comment: q = A r + beta q, p = r + beta p, p.q; then
// x, r update with r.r. Two kernels when the matrix has no long intervals
// (the SpMV carries the p / q update and p.q); otherwise the SpMV into w and
// an update kernel, then the x / r kernel.
template <class T, class A>
cudaError_t cg_iteration(const spc5_matrix* M, T* x, T* r, T* p, T* q, T* w, int64_t n, double* scal, A* part,
                         int nb, unsigned* ticket, cudaStream_t s) {
  cudaError_t e;
  if (M->nseg == 0 && M->I > 0) {
    if (M->vt == SPC5_F64)
      e = launch_fused_spmv_dot<F64>(M, r, p, q, part, ticket, scal, s);
    else if (M->vt == SPC5_F32)
      e = launch_fused_spmv_dot<F32>(M, r, p, q, part, ticket, scal, s);
    else
      e = launch_fused_spmv_dot<BF16>(M, r, p, q, part, ticket, scal, s);
  } else {
    e = spmv_any(M, r, w, s);
    if (e == cudaSuccess) k_cg_pq<T, A><<<nb, kThreads, 0, s>>>(p, q, r, w, n, scal, part, ticket);
  }
  if (e != cudaSuccess) return e;
  k_cg_xr_fused<T, A><<<nb, kThreads, 0, s>>>(x, r, p, q, n, scal, part, ticket);
  return cudaGetLastError();
}

// Runs CG iterations until sqrt(rho) <= stop or max_it; iteration body
// replayed from a CUDA graph when use_graph. Returns iterations done.
// `keep`: when not NULL the instantiated graph is taken from / left in *keep
// for later calls with the same vectors (the caller destroys it).
template <class T, class A>
spc5_status cg_loop(const spc5_matrix* M, T* x, T* r, T* p, T* q, T* w, int64_t n, double* scal, A* part, int nb,
                    unsigned* ticket, double stop, int max_it, int check_every, bool use_graph, double* host_scal,
                    cudaStream_t s, int* iters, cudaGraphExec_t* keep = nullptr) {
  cudaGraphExec_t exec = keep ? *keep : nullptr;
  if (use_graph && !exec) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cg: begin capture");
    cudaError_t e2 = cg_iteration<T, A>(M, x, r, p, q, w, n, scal, part, nb, ticket, s);
    e = cudaStreamEndCapture(s, &g);
    if (e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e2, "cg: capture");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cg: end capture");
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cg: instantiate");
  }
  // Residual checks: the first after check_every iterations; then the
  // observed convergence rate predicts how many more are needed, and the next
  // check is placed there (between 2 and 8 x check_every iterations away).
  int k = 0, next = check_every;
  double prev_norm = -1.0;
  int prev_k = 0;
  spc5_status st = SPC5_OK;
  while (k < max_it) {
    int batch = next;
    if (batch > max_it - k) batch = max_it - k;
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < batch && e == cudaSuccess; ++j)
      e = use_graph ? cudaGraphLaunch(exec, s) : cg_iteration<T, A>(M, x, r, p, q, w, n, scal, part, nb, ticket, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_scal, scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "cg: iteration");
      break;
    }
    k += batch;
    const double nr = sqrt(host_scal[S_RHO]);
    if (!(nr > stop)) break;  // also stops on NaN
    next = check_every;
    if (check_every > 1 && prev_norm > 0.0 && nr < prev_norm) {
      const double rate = log(nr / prev_norm) / (double)(k - prev_k);  // < 0
      const double need = log(stop / nr) / rate;
      int pred = (int)ceil(need);
      const int lo = check_every > 2 ? check_every / 4 : 1, hi = 8 * check_every;
      next = pred < lo ? lo : (pred > hi ? hi : pred);
    }
    prev_norm = nr;
    prev_k = k;
  }
  if (keep)
    *keep = exec;
  else if (exec)
    cudaGraphExecDestroy(exec);
  *iters = k;
  return st;
}

}  // namespace

spc5_status cg_impl(const spc5_matrix* A, const spc5_matrix* L, const double* b, double* x, const spc5_cg_opts* o,
                    spc5_cg_info* info, cudaStream_t user) {
  const int64_t n = A->n;
  // vector kernels: grid-stride, at most kVecBlocksPerSm CTAs per SM (each
  // CTA adds one partial and one ticket to the reductions)
  int64_t nb64 = (n + kThreads - 1) / kThreads;
  if (nb64 > (int64_t)sm_count() * kVecBlocksPerSm) nb64 = (int64_t)sm_count() * kVecBlocksPerSm;
  const int nb = nb64 > 0 ? (int)nb64 : 1;
  const double tol = o->tol > 0 ? o->tol : 1e-10;
  const int max_it = o->max_iters > 0 ? o->max_iters : 100000;
  const int max_outer = o->max_outer > 0 ? o->max_outer : 30;
  const double inner_tol = o->inner_tol > 0 ? o->inner_tol : 1e-6;
  const int inner_max = o->inner_max_iters > 0 ? o->inner_max_iters : 2000;
  const int every = o->check_every > 0 ? o->check_every : 8;
  const bool use_graph = o->use_graph != 0;

  // private stream ordered after the caller's work (capture needs a real stream)
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
  if (e != cudaSuccess) {
    if (s) cudaStreamDestroy(s);
    if (ev) cudaEventDestroy(ev);
    return cuda_fail(e, "cg: stream");
  }
  struct Cleanup {
    cudaStream_t s;
    cudaEvent_t ev;
    cudaStream_t user;
    ~Cleanup() {
      cudaEventRecord(ev, s);
      cudaStreamWaitEvent(user, ev, 0);
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
      cudaEventDestroy(ev);
    }
  } cleanup{s, ev, user};

  // partials: one per block of the widest grid (the fused SpMV: one lane per row)
  const int64_t nparts = (n + kThreads - 1) / kThreads + nb + 8;
  Buf scal_b, part_b, r_b, p_b, q_b, t_b, ticket_b;
  e = scal_b.alloc(sizeof(double) * S_COUNT);
  if (e == cudaSuccess) e = part_b.alloc(sizeof(double) * (size_t)nparts);
  if (e == cudaSuccess) e = ticket_b.alloc(sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(ticket_b.p, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = r_b.alloc(sizeof(double) * (size_t)n);
  if (e == cudaSuccess) e = p_b.alloc(sizeof(double) * (size_t)n);
  if (e == cudaSuccess) e = q_b.alloc(sizeof(double) * (size_t)n);
  if (e == cudaSuccess) e = t_b.alloc(sizeof(double) * (size_t)n);
  if (e != cudaSuccess) return cuda_fail(e, "cg: workspace");
  double* scal = (double*)scal_b.p;
  double* part = (double*)part_b.p;
  double* r = (double*)r_b.p;
  double* p = (double*)p_b.p;
  double* q = (double*)q_b.p;
  double* t = (double*)t_b.p;
  unsigned* ticket = (unsigned*)ticket_b.p;
  double hs[S_COUNT];
  e = cudaMemsetAsync(scal, 0, sizeof(double) * S_COUNT, s);
  if (e != cudaSuccess) return cuda_fail(e, "cg: init");

  // ||b||^2 into S_RHONEW's slot via a plain sum (b.b)
  k_dot_part<double, double><<<nb, kThreads, 0, s>>>(b, b, n, part);
  k_dot_final<double><<<1, kThreads, 0, s>>>(part, nb, scal, S_NORM);
  k_zero_vec<double><<<nb, kThreads, 0, s>>>(x, n);
  e = cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cg: norm of b");
  const double bnorm = sqrt(hs[S_NORM]);
  info->iterations = info->outer = info->inner_total = 0;
  info->converged = 0;
  info->rel_residual = 0.0;
  if (bnorm == 0.0) {  // x = 0 solves A x = 0
    info->converged = 1;
    return SPC5_OK;
  }
  const double stop = tol * bnorm;
  spc5_status st = SPC5_OK;
  if (!L) {
    // float64 CG from x = 0: r = b, p = q = 0, beta = 0 (scal cleared), rho = b.b
    k_copy_vec<double><<<nb, kThreads, 0, s>>>(r, b, n);
    k_zero_vec<double><<<nb, kThreads, 0, s>>>(p, n);
    k_zero_vec<double><<<nb, kThreads, 0, s>>>(q, n);
    k_dot_part<double, double><<<nb, kThreads, 0, s>>>(r, r, n, part);
    k_dot_final<double><<<1, kThreads, 0, s>>>(part, nb, scal, S_RHO);
    int it = 0;
    st = cg_loop<double, double>(A, x, r, p, q, t, n, scal, part, nb, ticket, stop, max_it, every, use_graph, hs, s,
                                 &it);
    info->iterations = it;
  } else if (o->reliable) {
    // float32 CG with reliable updates: one recurrence, never restarted; when
    // its residual norm has fallen by kReliableDelta since the last update,
    // x += x32 and r = b - A x in float64 replace the recurred quantities
    // (the search direction is kept, beta rescaled to the new residual)
    Buf r32_b, p32_b, q32_b, x32_b, w32_b, part32_b;
    e = r32_b.alloc(sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = p32_b.alloc(sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = q32_b.alloc(sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = x32_b.alloc(sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = w32_b.alloc(sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = part32_b.alloc(sizeof(float) * (size_t)nparts);
    if (e != cudaSuccess) return cuda_fail(e, "cg: workspace");
    float* r32 = (float*)r32_b.p;
    float* p32 = (float*)p32_b.p;
    float* q32 = (float*)q32_b.p;
    float* x32 = (float*)x32_b.p;
    float* w32 = (float*)w32_b.p;
    float* part32 = (float*)part32_b.p;
    // x = 0 (done), r = b; r32 = b, p32 = q32 = x32 = 0, beta = 0, rho = r32.r32
    k_copy_vec<double><<<nb, kThreads, 0, s>>>(r, b, n);
    k_narrow<<<nb, kThreads, 0, s>>>(b, r32, n);
    k_zero_vec<float><<<nb, kThreads, 0, s>>>(p32, n);
    k_zero_vec<float><<<nb, kThreads, 0, s>>>(q32, n);
    k_zero_vec<float><<<nb, kThreads, 0, s>>>(x32, n);
    k_dot_part<float, float><<<nb, kThreads, 0, s>>>(r32, r32, n, part32);
    k_dot_final<float><<<1, kThreads, 0, s>>>(part32, nb, scal, S_RHO);
    double rn_upd = bnorm;
    struct GraphKeep {
      cudaGraphExec_t g = nullptr;
      ~GraphKeep() {
        if (g) cudaGraphExecDestroy(g);
      }
    } keep;  // one captured iteration for all stretches between updates
    for (;;) {
      const double target = kReliableDelta * rn_upd > 0.5 * stop ? kReliableDelta * rn_upd : 0.5 * stop;
      int it = 0;
      st = cg_loop<float, float>(L, x32, r32, p32, q32, w32, n, scal, part32, nb, ticket, target,
                                 max_it - info->inner_total, every, use_graph, hs, s, &it, &keep.g);
      if (st != SPC5_OK) return st;
      info->inner_total += it;
      // reliable update in float64
      k_fold_x<<<nb, kThreads, 0, s>>>(x, x32, n);
      e = spmv_any(A, x, t, s);
      if (e != cudaSuccess) return cuda_fail(e, "cg: residual spmv");
      k_residual<<<nb, kThreads, 0, s>>>(r, b, t, n, part);
      k_dot_final<double><<<1, kThreads, 0, s>>>(part, nb, scal, S_NORM);
      e = cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(e, "cg: reliable update");
      info->outer += 1;
      const double rn = sqrt(hs[S_NORM]);
      if (!(rn > stop) || info->inner_total >= max_it || it == 0) break;
      rn_upd = rn;
      k_narrow<<<nb, kThreads, 0, s>>>(r, r32, n);
      k_dot_part<float, float><<<nb, kThreads, 0, s>>>(r32, r32, n, part32);
      k_dot_final<float><<<1, kThreads, 0, s>>>(part32, nb, scal, S_REPLACED);
    }
    info->iterations = info->inner_total;
  } else {
    Buf r32_b, p32_b, q32_b, x32_b, w32_b, part32_b;
    e = r32_b.alloc(sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = p32_b.alloc(sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = w32_b.alloc(sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = q32_b.alloc(sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = x32_b.alloc(sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = part32_b.alloc(sizeof(float) * (size_t)nparts);
    if (e != cudaSuccess) return cuda_fail(e, "cg: workspace");
    float* r32 = (float*)r32_b.p;
    float* p32 = (float*)p32_b.p;
    float* q32 = (float*)q32_b.p;
    float* x32 = (float*)x32_b.p;
    float* w32 = (float*)w32_b.p;
    float* part32 = (float*)part32_b.p;
    // r = b (x = 0)
    k_copy_vec<double><<<nb, kThreads, 0, s>>>(r, b, n);
    k_dot_part<double, double><<<nb, kThreads, 0, s>>>(r, r, n, part);
    k_dot_final<double><<<1, kThreads, 0, s>>>(part, nb, scal, S_NORM);
    for (int outer = 0; outer < max_outer; ++outer) {
      e = cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(e, "cg: residual norm");
      if (!(sqrt(hs[S_NORM]) > stop)) break;
      if (info->inner_total >= max_it) break;
      const double hs_norm = hs[S_NORM];
      // inner CG in float32 on A_low d = r / ||r||, from d = 0
      k_inner_start<<<nb, kThreads, 0, s>>>(r, r32, p32, q32, x32, n, scal);
      k_dot_part<float, float><<<nb, kThreads, 0, s>>>(r32, r32, n, part32);
      k_dot_final<float><<<1, kThreads, 0, s>>>(part32, nb, scal, S_RHO);
      e = cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(e, "cg: inner start");
      int it = 0;
      const int budget = inner_max < max_it - info->inner_total ? inner_max : max_it - info->inner_total;
      // solve only as far as the final tolerance needs: a relative reduction of
      // half of tol * ||b|| / ||r||, but never looser than inner_tol allows
      // from below (float32 cannot reach much further than about 1e-6)
      double itol = 0.5 * stop / sqrt(hs_norm);
      if (itol < inner_tol) itol = inner_tol;
      if (itol > 0.5) itol = 0.5;
      st = cg_loop<float, float>(L, x32, r32, p32, q32, w32, n, scal, part32, nb, ticket, itol * sqrt(hs[S_RHO]), budget,
                                 every, use_graph, hs, s, &it);
      if (st != SPC5_OK) return st;
      info->inner_total += it;
      // x += ||r|| d; r = b - A x in float64
      k_inner_apply<<<nb, kThreads, 0, s>>>(x, x32, n, scal);
      e = spmv_any(A, x, t, s);
      if (e != cudaSuccess) return cuda_fail(e, "cg: residual spmv");
      k_residual<<<nb, kThreads, 0, s>>>(r, b, t, n, part);
      k_dot_final<double><<<1, kThreads, 0, s>>>(part, nb, scal, S_NORM);
      info->outer = outer + 1;
    }
    info->iterations = info->inner_total;
  }
  if (st != SPC5_OK) return st;
  // true residual of the returned x, in float64
  e = spmv_any(A, x, t, s);
  if (e != cudaSuccess) return cuda_fail(e, "cg: final residual");
  k_residual<<<nb, kThreads, 0, s>>>(r, b, t, n, part);
  k_dot_final<double><<<1, kThreads, 0, s>>>(part, nb, scal, S_NORM);
  e = cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cg: final residual");
  info->rel_residual = sqrt(hs[S_NORM]) / bnorm;
  info->converged = info->rel_residual <= tol ? 1 : 0;
  return SPC5_OK;
}

}  // namespace spc5
