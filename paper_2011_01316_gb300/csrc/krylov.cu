// Krylov kernels: Gram-Schmidt passes of the Arnoldi process on the
// augmented matrix, the dense FP64 exponential of the projected Hessenberg
// matrix, and the vector combinations of the phi-sum (paper Sec. 2.3).
//
// Two storage forms share every kernel (template parameter FF):
//   FP64 form:   vectors are double arrays, arithmetic on the FP64 pipe.
//   mixed form:  vectors are float-float pairs (h, l); products and sums use
//                the error-free transformations of ff.cuh on the FP32 pipe,
//                which runs 74x faster than the FP64 pipe on this GPU.
// Reductions are deterministic: each block writes one partial per value, the
// last block to finish (atomic ticket) sums the partials in block order, one
// warp per value.
#include "common.cuh"
#include "ff.cuh"

namespace expdg {

namespace {

constexpr int RB = 2 * 152;     // blocks of the streaming reduction kernels
constexpr int NT = 256;         // threads per block
constexpr int NW = NT / 32;
constexpr int NORMS_MAX = 5;
constexpr int PHI_THREADS = 512;

template <bool FF>
struct Acc;
template <>
struct Acc<false> {
  using T = double;
  __device__ static T zero() { return 0.0; }
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static T shfl(T a, int off) { return __shfl_down_sync(0xffffffffu, a, off); }
  __device__ static double to_d(T a) { return a; }
};
template <>
struct Acc<true> {
  using T = ff;
  __device__ static T zero() { return ff{0.0f, 0.0f}; }
  __device__ static T add(T a, T b) { return ff_add(a, b); }
  __device__ static T shfl(T a, int off) { return ff_shfl_down(a, off); }
  __device__ static double to_d(T a) { return ff_to_double(a); }
};

template <bool FF>
__device__ __forceinline__ typename Acc<FF>::T load(const Vec& v, size_t i) {
  if constexpr (FF)
    return ff{v.h[i], v.l[i]};
  else
    return v.d[i];
}
template <bool FF>
__device__ __forceinline__ void store(const Vec& v, size_t i, typename Acc<FF>::T x) {
  if constexpr (FF) {
    v.h[i] = x.h;
    v.l[i] = x.l;
  } else {
    v.d[i] = x;
  }
}
// acc + a*b
template <bool FF>
__device__ __forceinline__ typename Acc<FF>::T fma_acc(typename Acc<FF>::T a, typename Acc<FF>::T b,
                                                      typename Acc<FF>::T acc) {
  if constexpr (FF)
    return ff_fma(a, b, acc);
  else
    return fma(a, b, acc);
}
template <bool FF>
__device__ __forceinline__ typename Acc<FF>::T from_d(double x) {
  if constexpr (FF)
    return ff_from_double(x);
  else
    return x;
}
template <bool FF>
__device__ __forceinline__ typename Acc<FF>::T negate(typename Acc<FF>::T x) {
  if constexpr (FF)
    return ff_neg(x);
  else
    return -x;
}

// Sum K per-thread values over the block; thread k < K of warp 0 gets total k.
template <bool FF, int K>
__device__ void block_sum(typename Acc<FF>::T (&v)[K], typename Acc<FF>::T* sh /* [NW][K] */) {
  using A = Acc<FF>;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    typename A::T x = v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = A::add(x, A::shfl(x, off));
    if (lane == 0) sh[w * K + k] = x;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    typename A::T x = A::zero();
    for (int ww = 0; ww < NW; ++ww) x = A::add(x, sh[ww * K + threadIdx.x]);
    v[threadIdx.x] = x;  // dynamic index on a register array: fine for small K
  }
}

// Ticket: true in the last block to arrive (after this block's partials are visible).
__device__ bool last_block(unsigned int* counter, unsigned int total) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == total - 1);
  __syncthreads();
  return am_last;
}

// In the last block: total_k = sum over g < G of part[k*G + g], k < K, one warp per k.
// Results to out[k] (double) by lane 0 of the owning warp.
template <bool FF>
__device__ void final_sums(const typename Acc<FF>::T* part, int K, int G, double* out) {
  using A = Acc<FF>;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < K; k += NW) {
    typename A::T x = A::zero();
    for (int g = lane; g < G; g += 32) {
      typename A::T pv;
      if constexpr (FF) {
        const float2 t = __ldcg(reinterpret_cast<const float2*>(part) + (size_t)k * G + g);
        pv = ff{t.x, t.y};
      } else {
        pv = __ldcg(part + (size_t)k * G + g);
      }
      x = A::add(x, pv);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = A::add(x, A::shfl(x, off));
    if (lane == 0) out[k] = A::to_d(x);
  }
}

struct LinArgs {
  Vec out;
  Vec x[NORMS_MAX];
  double a[NORMS_MAX];
  float ah[NORMS_MAX], al[NORMS_MAX];
  int nx;
  size_t n;
};

template <bool FF>
__global__ void __launch_bounds__(NT) k_lincomb(const LinArgs a) {
  using A = Acc<FF>;
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < a.n; i += (size_t)gridDim.x * NT) {
    typename A::T o = A::zero();
    for (int k = 0; k < a.nx; ++k) {
      const bool present = FF ? (a.x[k].h != nullptr) : (a.x[k].d != nullptr);
      if (!present) continue;
      typename A::T c;
      if constexpr (FF)
        c = ff{a.ah[k], a.al[k]};
      else
        c = a.a[k];
      o = fma_acc<FF>(c, load<FF>(a.x[k], i), o);
    }
    store<FF>(a.out, i, o);
  }
}

template <bool FF>
__global__ void __launch_bounds__(NT) k_norms(KState* ks, typename Acc<FF>::T* part, const LinArgs a) {
  using A = Acc<FF>;
  __shared__ typename A::T sh[NW * NORMS_MAX];
  typename A::T acc[NORMS_MAX];
#pragma unroll
  for (int k = 0; k < NORMS_MAX; ++k) acc[k] = A::zero();
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < a.n; i += (size_t)gridDim.x * NT) {
#pragma unroll
    for (int k = 0; k < NORMS_MAX; ++k) {
      if (k >= a.nx) break;
      const bool present = FF ? (a.x[k].h != nullptr) : (a.x[k].d != nullptr);
      if (!present) continue;
      typename A::T x = load<FF>(a.x[k], i);
      acc[k] = fma_acc<FF>(x, x, acc[k]);
    }
  }
  block_sum<FF, NORMS_MAX>(acc, sh);
  if (threadIdx.x < NORMS_MAX) part[threadIdx.x * gridDim.x + blockIdx.x] = acc[threadIdx.x];
  if (last_block(&ks->counter, gridDim.x)) {
    __shared__ double res[NORMS_MAX];
    final_sums<FF>(part, NORMS_MAX, gridDim.x, res);
    __syncthreads();
    if (threadIdx.x < NORMS_MAX) ks->red[threadIdx.x] = (threadIdx.x < a.nx) ? res[threadIdx.x] : 0.0;
    if (threadIdx.x == 0) ks->counter = 0;
  }
}

__global__ void k_to_f32(float* out, const double* x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = __double2float_rn(x[i]);
}
__global__ void k_f64_to_ff(Vec out, const double* x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    ff t = ff_from_double(x[i]);
    out.h[i] = t.h;
    out.l[i] = t.l;
  }
}
__global__ void k_ff_to_f64(double* out, Vec x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = ff_to_double(ff{x.h[i], x.l[i]});
}

template <bool FF>
__global__ void __launch_bounds__(NT) k_start(KState* ks, Vec u0, Vec b0, size_t N, int P, double eta,
                                             double beta) {
  using A = Acc<FF>;
  const bool present = FF ? (b0.h != nullptr) : (b0.d != nullptr);
  const size_t n_aug = N + P;
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n_aug; i += (size_t)gridDim.x * NT) {
    typename A::T x;
    if (i < N)
      x = present ? load<FF>(b0, i) : A::zero();
    else
      x = (i == n_aug - 1) ? from_d<FF>(1.0 / eta) : A::zero();
    store<FF>(u0, i, x);
  }
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < (MMAX + 1) * MMAX; k += NT) ks->H[k] = 0.0;
    if (threadIdx.x == 0) {
      const double s0 = 1.0 / beta;
      ks->s[0] = s0;
      ff t = ff_from_double(s0);
      ks->sh[0] = t.h;
      ks->sl[0] = t.l;
      ks->breakdown_at = 0;
      ks->accept = 0;
      ks->m_eff = 0;
      ks->err = 0.0;
      ks->wnorm0 = 0.0;
    }
  }
}

// grid: (gx, chunks); block (bx, c) handles basis vectors c*DOT_CHUNK .. +DOT_CHUNK-1.
template <bool FF>
__global__ void __launch_bounds__(NT) k_dots(KState* ks, typename Acc<FF>::T* part, Basis U, int J, size_t n_aug,
                                            int second) {
  using A = Acc<FF>;
  constexpr int K = DOT_CHUNK + 1;  // + ||w||^2 (first pass, chunk 0)
  __shared__ typename A::T sh[NW * K];
  const Vec w = U.at(J);
  const int c0 = blockIdx.y * DOT_CHUNK;
  const int nc = min(DOT_CHUNK, J - c0);
  Vec u[DOT_CHUNK];
#pragma unroll
  for (int c = 0; c < DOT_CHUNK; ++c) u[c] = U.at(c0 + (c < nc ? c : 0));
  typename A::T acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = A::zero();
  const bool wnorm = (!second) && blockIdx.y == 0;
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n_aug; i += (size_t)gridDim.x * NT) {
    const typename A::T wi = load<FF>(w, i);
#pragma unroll
    for (int c = 0; c < DOT_CHUNK; ++c)
      if (c < nc) acc[c] = fma_acc<FF>(load<FF>(u[c], i), wi, acc[c]);
    if (wnorm) acc[DOT_CHUNK] = fma_acc<FF>(wi, wi, acc[DOT_CHUNK]);
  }
  block_sum<FF, K>(acc, sh);
  const int G = gridDim.x;
  if (threadIdx.x < nc) part[(size_t)(c0 + threadIdx.x) * G + blockIdx.x] = acc[threadIdx.x];
  if (wnorm && threadIdx.x == DOT_CHUNK) part[(size_t)J * G + blockIdx.x] = acc[DOT_CHUNK];
  if (last_block(&ks->counter, gridDim.x * gridDim.y)) {
    __shared__ double res[MMAX + 1];
    final_sums<FF>(part, second ? J : J + 1, G, res);
    __syncthreads();
    const int j = J - 1;  // column of H being built
    for (int i = threadIdx.x; i < J; i += NT) {
      const double g = ks->s[i] * res[i];
      if (second) {
        ks->H[j * (MMAX + 1) + i] += g;
      } else {
        ks->H[j * (MMAX + 1) + i] = g;
      }
      ks->coef[i] = g * ks->s[i];
    }
    if (!second && threadIdx.x == 0) ks->wnorm0 = sqrt(res[J]);
    if (threadIdx.x == 0) ks->counter = 0;
  }
}

template <bool FF>
__global__ void __launch_bounds__(NT) k_update(KState* ks, typename Acc<FF>::T* part, Basis U, int J, size_t n_aug,
                                              int finish) {
  using A = Acc<FF>;
  __shared__ typename A::T cf[MMAX + 1];
  __shared__ typename A::T sh[NW];
  for (int i = threadIdx.x; i < J; i += NT) cf[i] = negate<FF>(from_d<FF>(ks->coef[i]));
  __syncthreads();
  const Vec w = U.at(J);
  typename A::T nrm[1] = {A::zero()};
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n_aug; i += (size_t)gridDim.x * NT) {
    typename A::T x = load<FF>(w, i);
    for (int k = 0; k < J; ++k) x = fma_acc<FF>(cf[k], load<FF>(U.at(k), i), x);
    store<FF>(w, i, x);
    if (finish) nrm[0] = fma_acc<FF>(x, x, nrm[0]);
  }
  if (!finish) return;
  block_sum<FF, 1>(nrm, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = nrm[0];
  if (last_block(&ks->counter, gridDim.x)) {
    __shared__ double res[1];
    final_sums<FF>(part, 1, gridDim.x, res);
    __syncthreads();
    if (threadIdx.x == 0) {
      const double h = sqrt(res[0]);
      const int j = J - 1;
      ks->H[j * (MMAX + 1) + J] = h;
      double s = 0.0;
      if (h <= 1e-13 * ks->wnorm0 || h == 0.0) {
        if (ks->breakdown_at == 0) ks->breakdown_at = J;
      } else {
        s = 1.0 / h;
      }
      ks->s[J] = s;
      ff t = ff_from_double(s);
      ks->sh[J] = t.h;
      ks->sl[J] = t.l;
      ks->counter = 0;
    }
  }
}

// Dense exponential of the m x m leading block of H by scaling and squaring
// of the degree-18 Taylor polynomial (Horner form), ||H / 2^s||_1 <= 1/2.
// One CTA, FP64, matrices in shared memory (row-major, leading dimension m).
__device__ void smem_matmul(const double* A, const double* B, double* C, int m) {
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx / m, c = idx - r * m;
    double s = 0.0;
    for (int k = 0; k < m; ++k) s = fma(A[r * m + k], B[k * m + c], s);
    C[idx] = s;
  }
}

__global__ void __launch_bounds__(PHI_THREADS) k_phi(KState* ks, int m_req, double beta, double tol, int force) {
  extern __shared__ double sm[];
  __shared__ int s_m;
  __shared__ double s_norm;
  if (threadIdx.x == 0) {
    const int b = ks->breakdown_at;
    s_m = (b > 0 && b < m_req) ? b : m_req;
  }
  __syncthreads();
  const int m = s_m;
  double* X = sm;
  double* E = X + m * m;
  double* T = E + m * m;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx / m, c = idx - r * m;
    X[idx] = ks->H[c * (MMAX + 1) + r];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double mx = 0.0;
    for (int c = threadIdx.x; c < m; c += 32) {
      double cs = 0.0;
      for (int r = 0; r < m; ++r) cs += fabs(X[r * m + c]);
      mx = fmax(mx, cs);
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    if (threadIdx.x == 0) s_norm = mx;
  }
  __syncthreads();
  int sq = 0;
  if (s_norm > 0.5) sq = (int)ceil(log2(s_norm / 0.5));
  const double scale = ldexp(1.0, -sq);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    X[idx] *= scale;
    const int r = idx / m, c = idx - r * m;
    E[idx] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = 18; k >= 1; --k) {
    smem_matmul(X, E, T, m);
    __syncthreads();
    const double inv = 1.0 / k;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int r = idx / m, c = idx - r * m;
      E[idx] = ((r == c) ? 1.0 : 0.0) + T[idx] * inv;
    }
    __syncthreads();
  }
  for (int k = 0; k < sq; ++k) {
    smem_matmul(E, E, T, m);
    __syncthreads();
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) E[idx] = T[idx];
    __syncthreads();
  }
  // y = E e_1 (first column)
  if (threadIdx.x == 0) {
    const bool brk = ks->breakdown_at > 0 && ks->breakdown_at <= m;
    const double hm = ks->H[(m - 1) * (MMAX + 1) + m];
    const double err = brk ? 0.0 : beta * hm * fabs(E[(m - 1) * m]);
    ks->err = err;
    ks->accept = (force || brk || err <= tol * beta) ? 1 : 0;
    ks->m_eff = m;
    ks->norm1 = s_norm;
    ks->squarings = sq;
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) ks->ycoef[i] = beta * E[i * m] * ks->s[i];
}

template <bool FF>
__global__ void __launch_bounds__(NT) k_combine(const KState* ks, Basis U, Vec base, Vec out, size_t N) {
  using A = Acc<FF>;
  __shared__ typename A::T cf[MMAX + 1];
  const int m = ks->m_eff;
  for (int i = threadIdx.x; i < m; i += NT) cf[i] = from_d<FF>(ks->ycoef[i]);
  __syncthreads();
  const bool base_d = base.d != nullptr, base_ff = base.h != nullptr;
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < N; i += (size_t)gridDim.x * NT) {
    typename A::T x = A::zero();
    for (int k = 0; k < m; ++k) x = fma_acc<FF>(cf[k], load<FF>(U.at(k), i), x);
    if (out.d != nullptr) {
      double o = A::to_d(x);
      if (base_d) o += base.d[i];
      if (base_ff) o += ff_to_double(ff{base.h[i], base.l[i]});
      out.d[i] = o;
    } else {
      ff o;
      if constexpr (FF)
        o = x;
      else
        o = ff_from_double(x);
      if (base_ff) o = ff_add(o, ff{base.h[i], base.l[i]});
      if (base_d) o = ff_add(o, ff_from_double(base.d[i]));
      out.h[i] = o.h;
      out.l[i] = o.l;
    }
  }
}

int grid_for(size_t n) {
  size_t b = (n + NT - 1) / NT;
  if (b > (size_t)RB) b = RB;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

size_t reduction_scratch_entries() { return (size_t)RB * (MMAX + 2) + 64; }

cudaError_t launch_lincomb(bool use_ff, Vec out, int nx, const Vec* x, const double* a, size_t n, cudaStream_t s) {
  if (nx > NORMS_MAX) return cudaErrorInvalidValue;
  LinArgs la{};
  la.out = out;
  la.nx = nx;
  la.n = n;
  for (int k = 0; k < nx; ++k) {
    la.x[k] = x[k];
    la.a[k] = a[k];
    la.ah[k] = (float)a[k];
    la.al[k] = (float)(a[k] - (double)la.ah[k]);
  }
  if (n == 0) return cudaSuccess;
  if (use_ff)
    k_lincomb<true><<<grid_for(n), NT, 0, s>>>(la);
  else
    k_lincomb<false><<<grid_for(n), NT, 0, s>>>(la);
  return cudaGetLastError();
}

cudaError_t launch_norms(bool use_ff, KState* ks, void* part, int nx, const Vec* x, size_t n, cudaStream_t s) {
  if (nx > NORMS_MAX) return cudaErrorInvalidValue;
  LinArgs la{};
  la.nx = nx;
  la.n = n;
  for (int k = 0; k < nx; ++k) la.x[k] = x[k];
  if (use_ff)
    k_norms<true><<<grid_for(n), NT, 0, s>>>(ks, static_cast<ff*>(part), la);
  else
    k_norms<false><<<grid_for(n), NT, 0, s>>>(ks, static_cast<double*>(part), la);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(float* out, const double* x, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_to_f32<<<grid_for(n), NT, 0, s>>>(out, x, n);
  return cudaGetLastError();
}
cudaError_t launch_f64_to_ff(Vec out, const double* x, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_f64_to_ff<<<grid_for(n), NT, 0, s>>>(out, x, n);
  return cudaGetLastError();
}
cudaError_t launch_ff_to_f64(double* out, Vec x, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_ff_to_f64<<<grid_for(n), NT, 0, s>>>(out, x, n);
  return cudaGetLastError();
}

cudaError_t launch_start(bool use_ff, KState* ks, Basis U, Vec b0, size_t N, int P, double eta, double beta,
                         cudaStream_t s) {
  const int g = grid_for(N + P);
  if (use_ff)
    k_start<true><<<g, NT, 0, s>>>(ks, U.at(0), b0, N, P, eta, beta);
  else
    k_start<false><<<g, NT, 0, s>>>(ks, U.at(0), b0, N, P, eta, beta);
  return cudaGetLastError();
}

cudaError_t launch_dots(bool use_ff, KState* ks, void* part, Basis U, int J, size_t n_aug, bool second, cudaStream_t s) {
  if (J < 1 || J > MMAX) return cudaErrorInvalidValue;
  const int chunks = (J + DOT_CHUNK - 1) / DOT_CHUNK;
  int gx = RB / chunks;
  const int need = (int)((n_aug + NT - 1) / NT);
  if (gx > need) gx = need;
  if (gx < 1) gx = 1;
  dim3 grid(gx, chunks);
  if (use_ff)
    k_dots<true><<<grid, NT, 0, s>>>(ks, static_cast<ff*>(part), U, J, n_aug, second ? 1 : 0);
  else
    k_dots<false><<<grid, NT, 0, s>>>(ks, static_cast<double*>(part), U, J, n_aug, second ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_update(bool use_ff, KState* ks, void* part, Basis U, int J, size_t n_aug, bool finish,
                          cudaStream_t s) {
  if (J < 1 || J > MMAX) return cudaErrorInvalidValue;
  const int g = grid_for(n_aug);
  if (use_ff)
    k_update<true><<<g, NT, 0, s>>>(ks, static_cast<ff*>(part), U, J, n_aug, finish ? 1 : 0);
  else
    k_update<false><<<g, NT, 0, s>>>(ks, static_cast<double*>(part), U, J, n_aug, finish ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_phi(KState* ks, int m, double beta, double tol, int force_accept, cudaStream_t s) {
  if (m < 1 || m > MMAX) return cudaErrorInvalidValue;
  const size_t smem = 3 * sizeof(double) * (size_t)m * m;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_phi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(3 * sizeof(double) * MMAX * MMAX));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_phi<<<1, PHI_THREADS, smem, s>>>(ks, m, beta, tol, force_accept);
  return cudaGetLastError();
}

cudaError_t launch_combine(bool use_ff, const KState* ks, Basis U, Vec base, Vec out, size_t N, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  if (use_ff)
    k_combine<true><<<grid_for(N), NT, 0, s>>>(ks, U, base, out, N);
  else
    k_combine<false><<<grid_for(N), NT, 0, s>>>(ks, U, base, out, N);
  return cudaGetLastError();
}

}  // namespace expdg
