// Krylov kernels: Gram-Schmidt passes of the Arnoldi process on the
// augmented matrix, the dense exponential of the projected Hessenberg matrix,
// and the vector combinations of the phi-sum (paper Sec. 2.3).
//
// Two storage forms share most kernels (template parameter FF):
//   FP64 storage:  vectors are double arrays, arithmetic on the FP64 pipe (the
//                  FP64 form, and the mixed form, whose basis vectors also keep
//                  an FP32 rounding in a shadow plane for the FP32 operator
//                  apply; its incomplete-orthogonalisation passes are the
//                  k_iom_*_mx kernels).
//   float-float:   vectors are float-float pairs (h, l); products and sums use
//                  the error-free transformations of ff.cuh on the FP32 pipe,
//                  which runs 74x faster than the FP64 pipe on this GPU.
// Reductions are deterministic: each block writes one partial per value and
// the partials are summed in block order, one warp per value - by the last
// block to finish (atomic ticket) in the full-orthogonalisation and norm
// kernels, by every block of the consuming launch in incomplete
// orthogonalisation (see there).
#include <algorithm>
#include <atomic>
#include <cooperative_groups.h>

#include "common.cuh"
#include "cvt.cuh"
#include "ff.cuh"
#include "fx.cuh"

namespace cg = cooperative_groups;

namespace expdg {

namespace {

// Blocks of the streaming reduction kernels: four per SM of the current
// device (red_blocks()), at most RB_MAX, which sizes the partial-sum scratch.
constexpr int RB_MAX = 1024;
constexpr int NT = 256;         // threads per block
constexpr int NW = NT / 32;
constexpr int NORMS_MAX = 5;

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
__device__ __forceinline__ typename Acc<FF>::T mul(typename Acc<FF>::T a, typename Acc<FF>::T b) {
  if constexpr (FF)
    return ff_mul(a, b);
  else
    return a * b;
}
template <bool FF>
__device__ __forceinline__ typename Acc<FF>::T negate(typename Acc<FF>::T x) {
  if constexpr (FF)
    return ff_neg(x);
  else
    return -x;
}

// Sum K per-thread values over the block; tot[k] (shared) receives total k.
template <bool FF, int K>
__device__ void block_sum(const typename Acc<FF>::T (&v)[K], typename Acc<FF>::T* sh /* [NW][K] */,
                          typename Acc<FF>::T* tot /* [K] */) {
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
    tot[threadIdx.x] = x;
  }
  __syncthreads();
}

// FP64 block sums for kernels whose main loop is bound by GB300's narrow FP64
// pipe, where an FP64 warp instruction costs the same whatever its active
// lanes: every thread's values go to shared memory and one warp adds them
// (NW - 1 additions a lane, then a five-step shuffle tree a value), instead of
// a shuffle tree in every warp (5 K FP64 warp instructions a warp).
template <int K>
__device__ void block_sum_1w(const double (&v)[K], double* sh /* [K][NT] */, double* tot /* [K] */) {
#pragma unroll
  for (int k = 0; k < K; ++k) sh[k * NT + threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double x = sh[k * NT + lane];
#pragma unroll
      for (int w = 1; w < NW; ++w) x += sh[k * NT + w * 32 + lane];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      if (lane == 0) tot[k] = x;
    }
  }
  __syncthreads();
}

// Element i of basis vector k.
template <bool FF>
__device__ __forceinline__ typename Acc<FF>::T ldb(const Basis& U, int k, size_t i) {
  const size_t o = (size_t)k * U.ld + i;
  if constexpr (FF)
    return ff{U.h[o], U.l[o]};
  else
    return U.d[o];
}
template <bool FF>
__device__ __forceinline__ void stb(const Basis& U, int k, size_t i, typename Acc<FF>::T x) {
  const size_t o = (size_t)k * U.ld + i;
  if constexpr (FF) {
    U.h[o] = x.h;
    U.l[o] = x.l;
  } else {
    U.d[o] = x;
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

// In the last block: total_k = sum over g < G of part[k*G + g], k < K.
// All K*G partials are first staged in shared memory `stage` (one coalesced
// load by every thread, so the L2 latency is paid once), then each warp sums
// its values from shared memory.  Results to out[k] (double).
template <bool FF>
__device__ void final_sums(const typename Acc<FF>::T* part, int K, int G, double* out,
                           typename Acc<FF>::T* stage) {
  using A = Acc<FF>;
  const int total = K * G;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    if constexpr (FF) {
      const float2 t = __ldcg(reinterpret_cast<const float2*>(part) + i);
      stage[i] = ff{t.x, t.y};
    } else {
      stage[i] = __ldcg(part + i);
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < K; k += NW) {
    typename A::T x = A::zero();
    for (int g = lane; g < G; g += 32) x = A::add(x, stage[k * G + g]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = A::add(x, A::shfl(x, off));
    if (lane == 0) out[k] = A::to_d(x);
  }
  __syncthreads();
}

// Dynamic shared memory of the reduction kernels (partial-sum staging).
template <bool FF>
__device__ __forceinline__ typename Acc<FF>::T* red_stage() {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  return reinterpret_cast<typename Acc<FF>::T*>(dyn_smem);
}

struct LinArgs {
  Vec out;
  Vec x[NORMS_MAX];
  double a[NORMS_MAX];
  float ah[NORMS_MAX], al[NORMS_MAX];
  int nx;
  size_t n;
  int dev_P;  // norms: also eta and beta of P augmentation vectors into KState (-1: no)
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
  __shared__ typename A::T tot[NORMS_MAX];
  block_sum<FF, NORMS_MAX>(acc, sh, tot);
  if (threadIdx.x < NORMS_MAX) part[threadIdx.x * gridDim.x + blockIdx.x] = tot[threadIdx.x];
  if (last_block(&ks->counter, gridDim.x)) {
    __shared__ double res[NORMS_MAX];
    final_sums<FF>(part, NORMS_MAX, gridDim.x, res, red_stage<FF>());
    __syncthreads();
    if (threadIdx.x < NORMS_MAX) ks->red[threadIdx.x] = (threadIdx.x < a.nx) ? res[threadIdx.x] : 0.0;
    if (threadIdx.x == 0) {
      if (a.dev_P >= 0) {
        double mx = 0.0;
        for (int i = 1; i <= a.dev_P; ++i) mx = fmax(mx, sqrt(res[i]));
        const double eta = tail_scale_of(mx);
        ks->eta = eta;
        ks->beta = sqrt(res[0] + (a.dev_P > 0 ? 1.0 / (eta * eta) : 0.0));
      }
      ks->counter = 0;
    }
  }
}

__global__ void k_to_f32(float* out, const double* x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = f64_to_f32_rn(x[i]);  // on the integer pipes
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
__global__ void __launch_bounds__(NT) k_start(KState* ks, Vec u0, Vec b0, size_t N, int P, double eta_in,
                                              double s0_in, double alpha, int mode) {
  // mode 1, 2: the sub-step's eta and beta come from the norms kernel
  const double eta = mode ? ks->eta : eta_in;
  const double beta = mode ? ks->beta : 0.0;
  const double s0 = mode == 1 ? (beta > 0.0 ? 1.0 / beta : 0.0) : (mode == 2 ? 1.0 : s0_in);
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
    if constexpr (!FF)
      if (u0.h != nullptr) u0.h[i] = f64_to_f32_rn(x);  // FP32 shadow (mixed form)
  }
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < (MMAX + 1) * MMAX; k += NT) ks->H[k] = 0.0;
    for (int k = threadIdx.x; k <= MMAX; k += NT) {
      const double v = (k == 0) ? s0 : 1.0;
      const ff f = ff_from_double(v);
      ks->vscale[k] = v;
      ks->vsf[k] = make_float2(f.h, f.l);
    }
    if (threadIdx.x == 0) {
      ks->jv.alpha = alpha;
      ks->jv.eta = eta;
      ks->jv.eta_f = (float)eta;
      ks->jv.alpha_h = (float)alpha;
      ks->jv.alpha_l = (float)(alpha - (double)(float)alpha);
      ks->breakdown_at = 0;
      ks->mprev = 0;
      ks->accept = 0;
      ks->m_eff = 0;
      ks->err = 0.0;
    }
  }
}

// Four consecutive elements of basis vector k starting at element 4g (vector
// bases are 256-byte aligned, so these are 16-byte loads).
template <bool FF>
struct Quad;
template <>
struct Quad<true> {
  ff v[4];
};
template <>
struct Quad<false> {
  double v[4];
};

template <bool FF>
__device__ __forceinline__ Quad<FF> ldq(const Basis& U, int k, size_t g) {
  Quad<FF> q;
  const size_t o = (size_t)k * U.ld + 4 * g;
  if constexpr (FF) {
    const float4 h = __ldg(reinterpret_cast<const float4*>(U.h + o));
    const float4 l = __ldg(reinterpret_cast<const float4*>(U.l + o));
    q.v[0] = ff{h.x, l.x};
    q.v[1] = ff{h.y, l.y};
    q.v[2] = ff{h.z, l.z};
    q.v[3] = ff{h.w, l.w};
  } else {
    const double2 a = __ldg(reinterpret_cast<const double2*>(U.d + o));
    const double2 b = __ldg(reinterpret_cast<const double2*>(U.d + o + 2));
    q.v[0] = a.x;
    q.v[1] = a.y;
    q.v[2] = b.x;
    q.v[3] = b.y;
  }
  return q;
}
template <bool FF>
__device__ __forceinline__ void stq(const Basis& U, int k, size_t g, const Quad<FF>& q) {
  const size_t o = (size_t)k * U.ld + 4 * g;
  if constexpr (FF) {
    *reinterpret_cast<float4*>(U.h + o) = make_float4(q.v[0].h, q.v[1].h, q.v[2].h, q.v[3].h);
    *reinterpret_cast<float4*>(U.l + o) = make_float4(q.v[0].l, q.v[1].l, q.v[2].l, q.v[3].l);
  } else {
    *reinterpret_cast<double2*>(U.d + o) = make_double2(q.v[0], q.v[1]);
    *reinterpret_cast<double2*>(U.d + o + 2) = make_double2(q.v[2], q.v[3]);
  }
}

// Last block of a DCGS2 dots launch: partial sums -> Hessenberg column j-1
// correction, column j, and the coefficients of the update pass.
template <bool FF>
__device__ void dots_last_block(KState* ks, const typename Acc<FF>::T* part, int j, int G) {
  const int nvec = j + 1;
    __shared__ double res[2 * MMAX + 4];
    __shared__ double sc[4];  // r, c
    final_sums<FF>(part, 2 * nvec + 1, G, res, red_stage<FF>());
    __syncthreads();
    // res[2i] = <x_i, u_j>, res[2i+1] = <x_i, w>; x_j = u_j; res[2 nvec] = <w, w>
    if (threadIdx.x == 0) {
      double ss = 0.0, sz = 0.0;
      for (int i = 0; i < j; ++i) {
        ss += res[2 * i] * res[2 * i];
        sz += res[2 * i] * res[2 * i + 1];
      }
      const double alpha = res[2 * j], gamma = res[2 * j + 1];
      const double r = sqrt(fmax(alpha - ss, 0.0));
      const double c = (r > 0.0) ? (gamma - sz) / r : 0.0;
      sc[0] = r;
      sc[1] = c;
      ks->inv_r = (r > 0.0) ? 1.0 / r : 0.0;
      ks->cu = (r > 0.0) ? c / r : 0.0;
      ks->wnorm = (r > 0.0) ? sqrt(res[2 * nvec]) / r : 0.0;
    }
    // stage columns 0..j-1 of H (rows 0..j) in shared memory: one coalesced load
    __shared__ double Hs[MMAX * (MMAX + 1)];
    for (int idx = threadIdx.x; idx < j * (MMAX + 1); idx += NT) Hs[idx] = ks->H[idx];
    __syncthreads();
    const double r = sc[0], c = sc[1];
    // column j-1: delayed re-orthogonalisation correction
    if (j >= 1) {
      for (int i = threadIdx.x; i < j; i += NT) {
        const double v = Hs[(j - 1) * (MMAX + 1) + i] + res[2 * i];
        Hs[(j - 1) * (MMAX + 1) + i] = v;
        ks->H[(j - 1) * (MMAX + 1) + i] = v;
      }
      if (threadIdx.x == 0) ks->H[(j - 1) * (MMAX + 1) + j] = r;
    }
    __syncthreads();
    // column j
    for (int k = threadIdx.x; k < j; k += NT) {
      double acc2 = 0.0;
      for (int i = (k > 0 ? k - 1 : 0); i < j; ++i) acc2 += res[2 * i] * Hs[i * (MMAX + 1) + k];
      ks->H[j * (MMAX + 1) + k] = (r > 0.0) ? (res[2 * k + 1] - acc2) / r : 0.0;
      ks->qcoef[k] = res[2 * k];
      ks->ucoef[k] = res[2 * k + 1] - ((r > 0.0) ? c / r : 0.0) * res[2 * k];
    }
    if (threadIdx.x == 0) {
      const double sjm1 = (j >= 1) ? res[2 * (j - 1)] : 0.0;
      ks->H[j * (MMAX + 1) + j] = (r > 0.0) ? (c - sjm1 * r) / r : 0.0;
      ks->counter = 0;
    }
}

// DCGS2 inner products of Arnoldi step j: grid (gx, chunks); block (bx, c)
// handles the vectors x_i, i = c*DOT_CHUNK .. +DOT_CHUNK-1 of [q_0..q_{j-1}, u_j],
// forming a_i = <x_i, u_j> and b_i = <x_i, w> (chunk 0 also <w, w>) over its
// share of the elements, four per thread with every load issued before the
// math.  The last block turns the sums into the Hessenberg entries and the
// coefficients of the update pass.
template <bool FF>
__global__ void __launch_bounds__(NT) k_dots(KState* ks, typename Acc<FF>::T* part, Basis U, int j, size_t n_aug) {
  griddep_wait();
  using A = Acc<FF>;
  constexpr int K = 2 * DOT_CHUNK + 1;
  __shared__ typename A::T sh[NW * K];
  __shared__ typename A::T tot[K];
  if (ks->breakdown_at > 0 && j >= ks->breakdown_at) return;  // uniform: every block leaves
  const int nvec = j + 1;
  const int c0 = blockIdx.y * DOT_CHUNK;
  const int nc = min(DOT_CHUNK, nvec - c0);
  typename A::T acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = A::zero();
  const bool wnorm = blockIdx.y == 0;
  const size_t ng = n_aug / 4;
  const size_t tid = blockIdx.x * (size_t)NT + threadIdx.x, nthr = (size_t)gridDim.x * NT;
  for (size_t g = tid; g < ng; g += nthr) {
    const Quad<FF> uj = ldq<FF>(U, j, g);
    const Quad<FF> w = ldq<FF>(U, j + 1, g);
    Quad<FF> x[DOT_CHUNK];
#pragma unroll
    for (int c = 0; c < DOT_CHUNK; ++c) x[c] = ldq<FF>(U, c0 + (c < nc ? c : 0), g);
#pragma unroll
    for (int c = 0; c < DOT_CHUNK; ++c)
      if (c < nc)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          acc[2 * c] = fma_acc<FF>(x[c].v[e], uj.v[e], acc[2 * c]);
          acc[2 * c + 1] = fma_acc<FF>(x[c].v[e], w.v[e], acc[2 * c + 1]);
        }
    if (wnorm)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[2 * DOT_CHUNK] = fma_acc<FF>(w.v[e], w.v[e], acc[2 * DOT_CHUNK]);
  }
  for (size_t i = 4 * ng + tid; i < n_aug; i += nthr) {
    const typename A::T ui = ldb<FF>(U, j, i), wi = ldb<FF>(U, j + 1, i);
    for (int c = 0; c < nc; ++c) {
      const typename A::T xi = ldb<FF>(U, c0 + c, i);
      acc[2 * c] = fma_acc<FF>(xi, ui, acc[2 * c]);
      acc[2 * c + 1] = fma_acc<FF>(xi, wi, acc[2 * c + 1]);
    }
    if (wnorm) acc[2 * DOT_CHUNK] = fma_acc<FF>(wi, wi, acc[2 * DOT_CHUNK]);
  }
  block_sum<FF, K>(acc, sh, tot);
  const int G = gridDim.x;
  if (threadIdx.x < 2 * nc) part[(size_t)(2 * c0 + threadIdx.x) * G + blockIdx.x] = tot[threadIdx.x];
  if (wnorm && threadIdx.x == 2 * DOT_CHUNK) part[(size_t)(2 * nvec) * G + blockIdx.x] = tot[2 * DOT_CHUNK];
  griddep_launch();
  if (last_block(&ks->counter, gridDim.x * gridDim.y)) dots_last_block<FF>(ks, part, j, G);
}

// DCGS2 update of Arnoldi step j (coefficients from k_dots):
//   q_j = (u_j - sum_k s_k q_k) / r                   -> slot j
//   u_{j+1} = (w - (c/r) u_j - sum_k (z_k - (c/r) s_k) q_k) / r -> slot j+1
// four elements per thread, two independent accumulation chains, and
// |u_{j+1}|^2 for the provisional H(j+1, j).
template <bool FF>
__global__ void __launch_bounds__(NT) k_update(KState* ks, typename Acc<FF>::T* part, Basis U, int j, size_t n_aug) {
  griddep_wait();
  using A = Acc<FF>;
  __shared__ typename A::T qc[MMAX + 1];
  __shared__ typename A::T uc[MMAX + 1];
  __shared__ typename A::T sc[2];
  __shared__ typename A::T sh[NW];
  if (ks->breakdown_at > 0 && j >= ks->breakdown_at) return;
  for (int k = threadIdx.x; k < j; k += NT) {
    qc[k] = negate<FF>(from_d<FF>(ks->qcoef[k]));
    uc[k] = negate<FF>(from_d<FF>(ks->ucoef[k]));
  }
  if (threadIdx.x == 0) {
    sc[0] = negate<FF>(from_d<FF>(ks->cu));
    sc[1] = from_d<FF>(ks->inv_r);
  }
  __syncthreads();
  const typename A::T ncu = sc[0], ir = sc[1];
  typename A::T nrm[1] = {A::zero()};
  const size_t ng = n_aug / 4;
  const size_t tid = blockIdx.x * (size_t)NT + threadIdx.x, nthr = (size_t)gridDim.x * NT;
  for (size_t g = tid; g < ng; g += nthr) {
    Quad<FF> xq = ldq<FF>(U, j, g);
    Quad<FF> xu = ldq<FF>(U, j + 1, g);
#pragma unroll
    for (int e = 0; e < 4; ++e) xu.v[e] = fma_acc<FF>(ncu, xq.v[e], xu.v[e]);
    for (int k = 0; k < j; ++k) {
      const Quad<FF> q = ldq<FF>(U, k, g);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        xq.v[e] = fma_acc<FF>(qc[k], q.v[e], xq.v[e]);
        xu.v[e] = fma_acc<FF>(uc[k], q.v[e], xu.v[e]);
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      xq.v[e] = mul<FF>(xq.v[e], ir);
      xu.v[e] = mul<FF>(xu.v[e], ir);
      nrm[0] = fma_acc<FF>(xu.v[e], xu.v[e], nrm[0]);
    }
    stq<FF>(U, j, g, xq);
    stq<FF>(U, j + 1, g, xu);
    if constexpr (!FF)
      if (U.h != nullptr)  // FP32 shadow of u_{j+1}, the next operator apply's input (mixed form)
        *reinterpret_cast<float4*>(U.h + (size_t)(j + 1) * U.ld + 4 * g) =
            make_float4(f64_to_f32_rn(xu.v[0]), f64_to_f32_rn(xu.v[1]), f64_to_f32_rn(xu.v[2]),
                        f64_to_f32_rn(xu.v[3]));
  }
  for (size_t i = 4 * ng + tid; i < n_aug; i += nthr) {
    typename A::T xq = ldb<FF>(U, j, i);
    typename A::T xu = fma_acc<FF>(ncu, xq, ldb<FF>(U, j + 1, i));
    for (int k = 0; k < j; ++k) {
      const typename A::T q = ldb<FF>(U, k, i);
      xq = fma_acc<FF>(qc[k], q, xq);
      xu = fma_acc<FF>(uc[k], q, xu);
    }
    xq = mul<FF>(xq, ir);
    xu = mul<FF>(xu, ir);
    nrm[0] = fma_acc<FF>(xu, xu, nrm[0]);
    stb<FF>(U, j, i, xq);
    stb<FF>(U, j + 1, i, xu);
    if constexpr (!FF)
      if (U.h != nullptr) U.h[(size_t)(j + 1) * U.ld + i] = f64_to_f32_rn(xu);
  }
  __shared__ typename A::T tot[1];
  block_sum<FF, 1>(nrm, sh, tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot[0];
  griddep_launch();
  if (last_block(&ks->counter, gridDim.x)) {
    __shared__ double res[1];
    final_sums<FF>(part, 1, gridDim.x, res, red_stage<FF>());
    __syncthreads();
    if (threadIdx.x == 0) {
      const double h = sqrt(res[0]);
      ks->H[j * (MMAX + 1) + j + 1] = h;
      if ((h <= 1e-13 * ks->wnorm || h == 0.0) && ks->breakdown_at == 0) ks->breakdown_at = j + 1;
      ks->counter = 0;
    }
  }
}


// ---- float-float (mixed form) Gram-Schmidt passes --------------------------
// Same mathematics as k_dots / k_update, with the products and sums done two
// elements at a time in packed FP32 (compensated accumulation, 12 packed
// instructions per two terms) so that the passes stay within the FP32 issue
// and pipe budget at HBM bandwidth.
constexpr int FF_CH = 2;  // basis vectors per block row

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

__global__ void __launch_bounds__(NT, 3) k_dots_ff(KState* ks, ff* part, Basis U, int j, size_t n_aug) {
  griddep_wait();
  constexpr int K = 2 * FF_CH + 1;
  __shared__ ff sh[NW * K];
  __shared__ ff tot[K];
  if (ks->breakdown_at > 0 && j >= ks->breakdown_at) return;
  const int nvec = j + 1;
  const int nch = (nvec + FF_CH - 1) / FF_CH;
  // consecutive blocks take the chunks of one element range, so u_j and w of
  // that range are read from HBM once and from L2 by the other chunks
  const int cy = blockIdx.x % nch, bx = blockIdx.x / nch, G = gridDim.x / nch;
  const int c0 = cy * FF_CH;
  const int nc = min(FF_CH, nvec - c0);
  const bool wnorm = cy == 0;
  float2 S[K], C[K];
#pragma unroll
  for (int k2 = 0; k2 < K; ++k2) S[k2] = C[k2] = make_float2(0.f, 0.f);
  const size_t ld = U.ld, ng = n_aug / 4;
  const float* __restrict__ Uh = U.h;
  const float* __restrict__ Ul = U.l;
  const size_t tid = bx * (size_t)NT + threadIdx.x, nthr = (size_t)G * NT;
  for (size_t g = tid; g < ng; g += nthr) {
    const size_t o = 4 * g;
    const float4 ujh = __ldg(reinterpret_cast<const float4*>(Uh + j * ld + o));
    const float4 ujl = __ldg(reinterpret_cast<const float4*>(Ul + j * ld + o));
    const float4 wh = __ldg(reinterpret_cast<const float4*>(Uh + (j + 1) * ld + o));
    const float4 wl = __ldg(reinterpret_cast<const float4*>(Ul + (j + 1) * ld + o));
    float4 xh[FF_CH], xl[FF_CH];
#pragma unroll
    for (int c = 0; c < FF_CH; ++c) {
      const size_t vo = (size_t)(c0 + (c < nc ? c : 0)) * ld + o;
      xh[c] = __ldg(reinterpret_cast<const float4*>(Uh + vo));
      xl[c] = __ldg(reinterpret_cast<const float4*>(Ul + vo));
    }
#pragma unroll
    for (int c = 0; c < FF_CH; ++c)
      if (c < nc) {
        dot2_acc(lo2(xh[c]), lo2(xl[c]), lo2(ujh), lo2(ujl), S[2 * c], C[2 * c]);
        dot2_acc(hi2(xh[c]), hi2(xl[c]), hi2(ujh), hi2(ujl), S[2 * c], C[2 * c]);
        dot2_acc(lo2(xh[c]), lo2(xl[c]), lo2(wh), lo2(wl), S[2 * c + 1], C[2 * c + 1]);
        dot2_acc(hi2(xh[c]), hi2(xl[c]), hi2(wh), hi2(wl), S[2 * c + 1], C[2 * c + 1]);
      }
    if (wnorm) {
      dot2_acc(lo2(wh), lo2(wl), lo2(wh), lo2(wl), S[2 * FF_CH], C[2 * FF_CH]);
      dot2_acc(hi2(wh), hi2(wl), hi2(wh), hi2(wl), S[2 * FF_CH], C[2 * FF_CH]);
    }
  }
  for (size_t i = 4 * ng + tid; i < n_aug; i += nthr) {  // ragged end, one element per lane pair
    const float2 ujh = make_float2(Uh[j * ld + i], 0.f), ujl = make_float2(Ul[j * ld + i], 0.f);
    const float2 wh = make_float2(Uh[(j + 1) * ld + i], 0.f), wl = make_float2(Ul[(j + 1) * ld + i], 0.f);
    for (int c = 0; c < nc; ++c) {
      const size_t vo = (size_t)(c0 + c) * ld + i;
      const float2 xh = make_float2(Uh[vo], 0.f), xl = make_float2(Ul[vo], 0.f);
      dot2_acc(xh, xl, ujh, ujl, S[2 * c], C[2 * c]);
      dot2_acc(xh, xl, wh, wl, S[2 * c + 1], C[2 * c + 1]);
    }
    if (wnorm) dot2_acc(wh, wl, wh, wl, S[2 * FF_CH], C[2 * FF_CH]);
  }
  ff v[K];
#pragma unroll
  for (int k2 = 0; k2 < K; ++k2) v[k2] = dot2_value(S[k2], C[k2]);
  block_sum<true, K>(v, sh, tot);
  if (threadIdx.x < 2 * nc) part[(size_t)(2 * c0 + threadIdx.x) * G + bx] = tot[threadIdx.x];
  if (wnorm && threadIdx.x == 2 * FF_CH) part[(size_t)(2 * nvec) * G + bx] = tot[2 * FF_CH];
  griddep_launch();
  if (last_block(&ks->counter, gridDim.x)) dots_last_block<true>(ks, part, j, G);
}

constexpr int UKG = 4;         // thread groups sharing one quad's basis loop
constexpr int UQB = NT / UKG;  // quads per block tile

// Update pass, float-float form.  A block tile is UQB quads (four elements
// each); the UKG thread groups of the block split the basis vectors of every
// quad (k = group, group + UKG, ...) so each quad has UKG independent load
// chains, and group 0 adds the other groups' partial sums from shared memory,
// scales, stores q_j and u_{j+1} and accumulates |u_{j+1}|^2.
__global__ void __launch_bounds__(NT, 3) k_update_ff(KState* ks, ff* part, Basis U, int j, size_t n_aug) {
  griddep_wait();
  __shared__ float2 qc[MMAX + 1];  // (h, l) of -s_k
  __shared__ float2 uc[MMAX + 1];  // (h, l) of -(z_k - (c/r) s_k)
  __shared__ float2 sc[2];         // -(c/r), 1/r
  __shared__ float4 xs[UKG][4][UQB];  // every group's partial sums of the tile
  __shared__ ff sh[NW];
  if (ks->breakdown_at > 0 && j >= ks->breakdown_at) return;
  for (int k2 = threadIdx.x; k2 < j; k2 += NT) {
    const ff a = ff_from_double(-ks->qcoef[k2]);
    const ff b = ff_from_double(-ks->ucoef[k2]);
    qc[k2] = make_float2(a.h, a.l);
    uc[k2] = make_float2(b.h, b.l);
  }
  if (threadIdx.x == 0) {
    const ff a = ff_from_double(-ks->cu), b = ff_from_double(ks->inv_r);
    sc[0] = make_float2(a.h, a.l);
    sc[1] = make_float2(b.h, b.l);
  }
  __syncthreads();
  const float2 ncu_h = make_float2(sc[0].x, sc[0].x), ncu_l = make_float2(sc[0].y, sc[0].y);
  const float2 ir_h = make_float2(sc[1].x, sc[1].x), ir_l = make_float2(sc[1].y, sc[1].y);
  const int qi = threadIdx.x % UQB, grp = threadIdx.x / UQB;
  float2 S = make_float2(0.f, 0.f), C = make_float2(0.f, 0.f);
  const size_t ld = U.ld, ng = n_aug / 4;
  float* __restrict__ Uh = U.h;
  float* __restrict__ Ul = U.l;
  const float2 z2 = make_float2(0.f, 0.f);
  for (size_t tile = blockIdx.x; tile * UQB < ng; tile += gridDim.x) {
    const size_t g = tile * UQB + qi;
    const bool valid = g < ng;
    const size_t o = 4 * g;
    float2 qh0 = z2, qh1 = z2, ql0 = z2, ql1 = z2, uh0 = z2, uh1 = z2, ul0 = z2, ul1 = z2;
    if (valid) {
      if (grp == 0) {
        const float4 ujh = *reinterpret_cast<const float4*>(Uh + j * ld + o);
        const float4 ujl = *reinterpret_cast<const float4*>(Ul + j * ld + o);
        const float4 wh = *reinterpret_cast<const float4*>(Uh + (j + 1) * ld + o);
        const float4 wl = *reinterpret_cast<const float4*>(Ul + (j + 1) * ld + o);
        qh0 = lo2(ujh), qh1 = hi2(ujh), ql0 = lo2(ujl), ql1 = hi2(ujl);
        uh0 = lo2(wh), uh1 = hi2(wh), ul0 = lo2(wl), ul1 = hi2(wl);
        axpy2_acc(ncu_h, ncu_l, lo2(ujh), lo2(ujl), uh0, ul0);
        axpy2_acc(ncu_h, ncu_l, hi2(ujh), hi2(ujl), uh1, ul1);
      }
      int cnt = 0;
      // one basis quad in flight ahead of the arithmetic
      float4 nh = make_float4(0.f, 0.f, 0.f, 0.f), nl = nh;
      if (grp < j) {
        nh = __ldg(reinterpret_cast<const float4*>(Uh + (size_t)grp * ld + o));
        nl = __ldg(reinterpret_cast<const float4*>(Ul + (size_t)grp * ld + o));
      }
      for (int k2 = grp; k2 < j; k2 += UKG, ++cnt) {
        const float4 bh = nh, bl = nl;
        if (k2 + UKG < j) {
          nh = __ldg(reinterpret_cast<const float4*>(Uh + (size_t)(k2 + UKG) * ld + o));
          nl = __ldg(reinterpret_cast<const float4*>(Ul + (size_t)(k2 + UKG) * ld + o));
        }
        const float2 a = qc[k2], b = uc[k2];
        const float2 ah = make_float2(a.x, a.x), al = make_float2(a.y, a.y);
        const float2 bhh = make_float2(b.x, b.x), bll = make_float2(b.y, b.y);
        axpy2_acc(ah, al, lo2(bh), lo2(bl), qh0, ql0);
        axpy2_acc(ah, al, hi2(bh), hi2(bl), qh1, ql1);
        axpy2_acc(bhh, bll, lo2(bh), lo2(bl), uh0, ul0);
        axpy2_acc(bhh, bll, hi2(bh), hi2(bl), uh1, ul1);
        if ((cnt & 15) == 15) {
          ff2_norm(qh0, ql0);
          ff2_norm(qh1, ql1);
          ff2_norm(uh0, ul0);
          ff2_norm(uh1, ul1);
        }
      }
      ff2_norm(qh0, ql0);
      ff2_norm(qh1, ql1);
      ff2_norm(uh0, ul0);
      ff2_norm(uh1, ul1);
    }
    xs[grp][0][qi] = make_float4(qh0.x, qh0.y, qh1.x, qh1.y);
    xs[grp][1][qi] = make_float4(ql0.x, ql0.y, ql1.x, ql1.y);
    xs[grp][2][qi] = make_float4(uh0.x, uh0.y, uh1.x, uh1.y);
    xs[grp][3][qi] = make_float4(ul0.x, ul0.y, ul1.x, ul1.y);
    __syncthreads();
    {
      // thread t finalises element t of the tile: quad t/4, lane t%4
      const int eq = threadIdx.x >> 2, el = threadIdx.x & 3;
      const size_t ge = tile * UQB + eq;
      if (ge < ng) {
        auto pick = [&](const float4& v) { return el == 0 ? v.x : el == 1 ? v.y : el == 2 ? v.z : v.w; };
        ff xq{0.f, 0.f}, xu{0.f, 0.f};
#pragma unroll
        for (int gg = 0; gg < UKG; ++gg) {
          xq = ff_add(xq, ff{pick(xs[gg][0][eq]), pick(xs[gg][1][eq])});
          xu = ff_add(xu, ff{pick(xs[gg][2][eq]), pick(xs[gg][3][eq])});
        }
        const ff ir{sc[1].x, sc[1].y};
        xq = ff_mul(xq, ir);
        xu = ff_mul(xu, ir);
        dot2_acc(make_float2(xu.h, 0.f), make_float2(xu.l, 0.f), make_float2(xu.h, 0.f), make_float2(xu.l, 0.f), S, C);
        const size_t i = 4 * ge + el;
        Uh[j * ld + i] = xq.h;
        Ul[j * ld + i] = xq.l;
        Uh[(j + 1) * ld + i] = xu.h;
        Ul[(j + 1) * ld + i] = xu.l;
      }
    }
    __syncthreads();  // xs is reused by the next tile
  }
  const size_t tid = blockIdx.x * (size_t)NT + threadIdx.x, nthr = (size_t)gridDim.x * NT;
  for (size_t i = 4 * ng + tid; i < n_aug; i += nthr) {  // ragged end
    ff xq{Uh[j * ld + i], Ul[j * ld + i]};
    ff xu = ff_fma(ff{sc[0].x, sc[0].y}, xq, ff{Uh[(j + 1) * ld + i], Ul[(j + 1) * ld + i]});
    for (int k2 = 0; k2 < j; ++k2) {
      const ff q{Uh[k2 * ld + i], Ul[k2 * ld + i]};
      xq = ff_fma(ff{qc[k2].x, qc[k2].y}, q, xq);
      xu = ff_fma(ff{uc[k2].x, uc[k2].y}, q, xu);
    }
    const ff ir{sc[1].x, sc[1].y};
    xq = ff_mul(xq, ir);
    xu = ff_mul(xu, ir);
    dot2_acc(make_float2(xu.h, 0.f), make_float2(xu.l, 0.f), make_float2(xu.h, 0.f), make_float2(xu.l, 0.f), S, C);
    Uh[j * ld + i] = xq.h;
    Ul[j * ld + i] = xq.l;
    Uh[(j + 1) * ld + i] = xu.h;
    Ul[(j + 1) * ld + i] = xu.l;
  }
  ff v[1] = {dot2_value(S, C)};
  __shared__ ff tot[1];
  block_sum<true, 1>(v, sh, tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot[0];
  griddep_launch();
  if (last_block(&ks->counter, gridDim.x)) {
    __shared__ double res[1];
    final_sums<true>(part, 1, gridDim.x, res, red_stage<true>());
    __syncthreads();
    if (threadIdx.x == 0) {
      const double h = sqrt(res[0]);
      ks->H[j * (MMAX + 1) + j + 1] = h;
      if ((h <= 1e-13 * ks->wnorm || h == 0.0) && ks->breakdown_at == 0) ks->breakdown_at = j + 1;
      ks->counter = 0;
    }
  }
}

// ---- incomplete orthogonalisation (KIOPS's replacement for Arnoldi, Sec. 1) ----
// Window of the last KW basis vectors.  Slot i holds an unnormalised vector,
// v_i = c_i slot_i with c_i = 1 / ||slot_i||, so the normalisation costs no
// pass: the operator apply of step j takes slot_j as it is (w' = A_hat
// slot_j = w / c_j), the update stores the unnormalised residual vector
// slot_{j+1} = w_new = w - sum h_{i,j} v_i (so ||slot_{j+1}|| = h_{j+1,j}
// stays the size of A_hat: no product of subdiagonals builds up in FP32),
// and the final combination folds c_i into its coefficients.  The window vectors are
// mutually orthogonal in exact arithmetic, so one classical pass (all window
// products at once, then one update) equals the modified sweep.
//
// No launch of a step ends with a last-block reduction (a fence, a ticket and
// one block summing every partial while the GPU idles): the window-products
// launch only writes its per-block partial sums, and every block of the
// update launch sums them itself, in the same order, so all blocks derive the
// same coefficients; the update launch likewise leaves the partials of
// ||slot_{j+1}||^2 to the next update launch (or to the phi kernel at a check).
//
// Loads before griddepcontrol.wait.  Every launch of an Arnoldi step calls
// griddepcontrol.launch_dependents only after its own griddepcontrol.wait,
// so when a launch is scheduled every launch before its immediate
// predecessor has completed (and a segment starts after a plain launch).  A
// launch may therefore read before the wait what those earlier launches
// wrote: the window-products launch the window slots (last written by the
// previous update), the update launch w' and the window slots (the operator
// apply and the previous update); only its predecessor's output waits.
constexpr int IOP_MAX = EXPDG_MAX_IOP;
// The update launches' norm partials follow the window products' partials in
// the reduction scratch: two regions, by the parity of j.
constexpr int IOM_UPD_OFF = (IOP_MAX + 1) * RB_MAX;

// Prologue of update launch j (FP64 form; the float-float form uses
// iom_prologue_ff below), in every block: sums the window products of
// launch j (<slot_i, w'> for the window, then |w'|^2) and ||slot_j||^2 (the
// partials of update launch j - 1), then
//   c_j = 1 / ||slot_j||  (c_0: set by the start kernel),
//   h_{j,j-1} = ||slot_j||, a breakdown when ||slot_j|| <= 1e-13 ||w_{j-1}||,
//   h_{i,j} = c_i c_j <slot_i, w'>,
// and the update slot_{j+1} = c_j w' + sum_i coef_i slot_i with
//   coef_i = -c_j c_i^2 <slot_i, w'>.
// Block 0 stores c_j, the H entries and ||w_j|| = c_j ||w'||.  Returns false
// on a breakdown at j (then there is nothing to update).
template <bool FF>
__device__ bool iom_prologue(KState* ks, const typename Acc<FF>::T* part, int j, int lo, int nwin, int K, int Gd,
                             int Gu, double* coef /* shared, [IOP_MAX] */, double* cjs /* shared */) {
  using A = Acc<FF>;
  using T = typename A::T;
  T* stage = red_stage<FF>();
  __shared__ double res[IOP_MAX + 2];
  __shared__ double cw[IOP_MAX];  // c_i of the window (c_j: computed below)
  __shared__ double s_c0, s_wprev;
  __shared__ int s_ok;
  // every global load first (one round trip): partials, window scales, flags
  const int nd = K * Gd, nu = (j > 0) ? Gu : 0;
  const T* pu = part + IOM_UPD_OFF + ((j + 1) & 1) * RB_MAX;  // region of launch j - 1
  for (int i = threadIdx.x; i < nd + nu; i += blockDim.x) {
    const T* src = (i < nd) ? part + i : pu + (i - nd);
    if constexpr (FF) {
      const float2 t = __ldcg(reinterpret_cast<const float2*>(src));
      stage[i] = ff{t.x, t.y};
    } else {
      stage[i] = __ldcg(src);
    }
  }
  if ((int)threadIdx.x < nwin) cw[threadIdx.x] = __ldcg(&ks->vscale[lo + threadIdx.x]);
  if (threadIdx.x == 32) {
    const int b = __ldcg(&ks->breakdown_at);
    s_ok = (b > 0 && j >= b) ? 0 : 1;  // an earlier breakdown: nothing to do
    s_c0 = __ldcg(&ks->vscale[0]);
    s_wprev = __ldcg(&ks->wnp[(j + 1) & 1]);
  }
  __syncthreads();
  if (!s_ok) return false;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int rows = K + (j > 0 ? 1 : 0);
  for (int k = w; k < rows; k += NW) {
    const T* row = (k < K) ? stage + k * Gd : stage + nd;
    const int G = (k < K) ? Gd : Gu;
    T x = A::zero();
    for (int g = lane; g < G; g += 32) x = A::add(x, row[g]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = A::add(x, A::shfl(x, off));
    if (lane == 0) res[k] = A::to_d(x);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = true;
    double cj = s_c0;
    if (j > 0) {
      const double ns = sqrt(res[K]);
      ok = !(ns <= 1e-13 * s_wprev || ns == 0.0);
      cj = (ns > 0.0) ? 1.0 / ns : 0.0;
      if (blockIdx.x == 0) {
        ks->H[(j - 1) * (MMAX + 1) + j] = ns;
        ks->vscale[j] = cj;
        if (!ok && ks->breakdown_at == 0) ks->breakdown_at = j;
      }
    }
    if (ok) {
      for (int c = 0; c < nwin; ++c) {
        const int i = lo + c;
        const double ci = (i == j) ? cj : cw[c];
        coef[c] = -cj * ci * ci * res[c];
        if (blockIdx.x == 0) ks->H[j * (MMAX + 1) + i] = ci * cj * res[c];
      }
      if (blockIdx.x == 0) ks->wnp[j & 1] = cj * sqrt(res[K - 1]);
    }
    *cjs = cj;
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Float-float form of iom_prologue: the same quantities, with every scalar
// operation on the FP32 pipe (fx arithmetic: Dekker division and square
// root), so the update's critical path carries no FP64 instruction (on GB300
// one FP64 warp instruction holds the narrow FP64 pipe for tens of cycles,
// active lanes or not).  cf[c] = coef_c as (h, l).  The FP64 copies for the
// phi kernel (H entries, vscale_j, ||w_j||) are written after the update, one
// item per block, by write_iom_scalars.
struct IomScalars {
  fx h[IOP_MAX];  // H(lo + c, j)
  fx hsub;        // H(j, j-1) = ||slot_j||
  fx cj;          // c_j
  fx wn;          // ||w_j|| = c_j ||w'||
  int ok;
};
// Returns -1 after an earlier breakdown (nothing to do), 0 on a breakdown at
// j (to be recorded), 1 to update.
__device__ int iom_prologue_ff(KState* ks, const ff* part, int j, int lo, int nwin, int K, int Gd, int Gu,
                               float2* cf /* shared, [IOP_MAX] */, IomScalars* sc /* shared */) {
  ff* stage = red_stage<true>();
  __shared__ ff res[IOP_MAX + 2];
  __shared__ float2 cw[IOP_MAX];  // c_i of the window (c_j: computed below)
  __shared__ float2 s_c0;
  __shared__ float s_wprev;
  __shared__ int s_go;
  const int nd = K * Gd, nu = (j > 0) ? Gu : 0;
  const ff* pu = part + IOM_UPD_OFF + ((j + 1) & 1) * RB_MAX;  // region of launch j - 1
  for (int i = threadIdx.x; i < nd + nu; i += blockDim.x) {
    const ff* src = (i < nd) ? part + i : pu + (i - nd);
    const float2 t = __ldcg(reinterpret_cast<const float2*>(src));
    stage[i] = ff{t.x, t.y};
  }
  if ((int)threadIdx.x < nwin) cw[threadIdx.x] = __ldcg(&ks->vsf[lo + threadIdx.x]);
  if (threadIdx.x == 32) {
    const int b = __ldcg(&ks->breakdown_at);
    s_go = (b > 0 && j >= b) ? 0 : 1;  // an earlier breakdown: nothing to do
    s_c0 = __ldcg(&ks->vsf[0]);
    s_wprev = (float)__ldcg(&ks->wnp[(j + 1) & 1]);
  }
  __syncthreads();
  if (!s_go) return -1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int rows = K + (j > 0 ? 1 : 0);
  for (int k = w; k < rows; k += NW) {
    const ff* row = (k < K) ? stage + k * Gd : stage + nd;
    const int G = (k < K) ? Gd : Gu;
    ff x{0.0f, 0.0f};
    for (int g = lane; g < G; g += 32) x = ff_add(x, row[g]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = ff_add(x, ff_shfl_down(x, off));
    if (lane == 0) res[k] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = true;
    fx cj(s_c0.x, s_c0.y), ns(0.0f, 0.0f);
    if (j > 0) {
      ns = sqrt(fx(res[K]));
      ok = !(ns.h <= 1e-13f * s_wprev || ns.h == 0.0f);
      cj = (ns.h > 0.0f) ? fx(1.0f) / ns : fx(0.0f, 0.0f);
    }
    sc->hsub = ns;
    sc->cj = cj;
    sc->wn = cj * sqrt(fx(res[K - 1]));
    sc->ok = ok ? 1 : 0;
    if (ok)
      for (int c = 0; c < nwin; ++c) {
        const int i = lo + c;
        const fx ci = (i == j) ? cj : fx(cw[c].x, cw[c].y);
        const fx h = ci * cj * fx(res[c]);
        sc->h[c] = h;
        const fx co = -(h * ci);
        cf[c] = make_float2(co.h, co.l);
      }
  }
  __syncthreads();
  return sc->ok;
}

// The update's FP64 results for the phi kernel and the next launches, one item
// per block (item k by block k mod gridDim.x): vscale_j (and its pair),
// breakdown_at, H(j, j-1), ||w_j||, H(lo + c, j).
__device__ void write_iom_scalars(KState* ks, const IomScalars& sc, int j, int lo, int nwin) {
  if (threadIdx.x != 0) return;
  const int items = 3 + nwin;
  for (int k = blockIdx.x; k < items; k += gridDim.x) {
    if (k == 0) {
      if (j > 0) {
        ks->vscale[j] = (double)sc.cj.h + (double)sc.cj.l;
        ks->vsf[j] = make_float2(sc.cj.h, sc.cj.l);
        if (!sc.ok && ks->breakdown_at == 0) ks->breakdown_at = j;
      }
    } else if (k == 1) {
      if (j > 0) ks->H[(j - 1) * (MMAX + 1) + j] = (double)sc.hsub.h + (double)sc.hsub.l;
    } else if (k == 2) {
      if (sc.ok) ks->wnp[j & 1] = (double)sc.wn.h + (double)sc.wn.l;
    } else if (sc.ok) {
      const int c = k - 3;
      ks->H[j * (MMAX + 1) + lo + c] = (double)sc.h[c].h + (double)sc.h[c].l;
    }
  }
}

// Float-float form: packed compensated products, four elements per thread
// per trip, every load of a trip issued before the arithmetic.
template <int KW>
__global__ void __launch_bounds__(NT) k_iom_dots_ff(KState* ks, ff* part, Basis U, int j, size_t n_aug) {
  constexpr int K = KW + 1;
  __shared__ ff sh[NW * K];
  __shared__ ff tot[K];
  // (after a breakdown these partials are never read: no flag check up front)
  const int lo = max(0, j - KW + 1), nwin = j - lo + 1;
  float2 S[K], C[K];
#pragma unroll
  for (int k = 0; k < K; ++k) S[k] = C[k] = make_float2(0.f, 0.f);
  const size_t ld = U.ld, ng = n_aug / 4;
  const float* __restrict__ Uh = U.h;
  const float* __restrict__ Ul = U.l;
  const size_t tid = blockIdx.x * (size_t)NT + threadIdx.x, nthr = (size_t)gridDim.x * NT;
  // the first trip's window slots before the wait (see above), w' after it
  float4 pxh[KW], pxl[KW];
  if (tid < ng) {
#pragma unroll
    for (int c = 0; c < KW; ++c) {
      const size_t vo = (size_t)(lo + (c < nwin ? c : 0)) * ld + 4 * tid;
      pxh[c] = __ldg(reinterpret_cast<const float4*>(Uh + vo));
      pxl[c] = __ldg(reinterpret_cast<const float4*>(Ul + vo));
    }
  }
  griddep_wait();
  for (size_t g = tid; g < ng; g += nthr) {
    const size_t o = 4 * g;
    const float4 wh = __ldg(reinterpret_cast<const float4*>(Uh + (j + 1) * ld + o));
    const float4 wl = __ldg(reinterpret_cast<const float4*>(Ul + (j + 1) * ld + o));
    float4 xh[KW], xl[KW];
#pragma unroll
    for (int c = 0; c < KW; ++c) {
      if (g == tid) {
        xh[c] = pxh[c];
        xl[c] = pxl[c];
      } else {
        const size_t vo = (size_t)(lo + (c < nwin ? c : 0)) * ld + o;
        xh[c] = __ldg(reinterpret_cast<const float4*>(Uh + vo));
        xl[c] = __ldg(reinterpret_cast<const float4*>(Ul + vo));
      }
    }
#pragma unroll
    for (int c = 0; c < KW; ++c)
      if (c < nwin) {
        dot2_acc(lo2(xh[c]), lo2(xl[c]), lo2(wh), lo2(wl), S[c], C[c]);
        dot2_acc(hi2(xh[c]), hi2(xl[c]), hi2(wh), hi2(wl), S[c], C[c]);
      }
    dot2_acc(lo2(wh), lo2(wl), lo2(wh), lo2(wl), S[KW], C[KW]);
    dot2_acc(hi2(wh), hi2(wl), hi2(wh), hi2(wl), S[KW], C[KW]);
  }
  for (size_t i = 4 * ng + tid; i < n_aug; i += nthr) {  // ragged end
    const float2 wh = make_float2(Uh[(j + 1) * ld + i], 0.f), wl = make_float2(Ul[(j + 1) * ld + i], 0.f);
#pragma unroll
    for (int c = 0; c < KW; ++c)  // constant indices keep S, C in registers
      if (c < nwin) {
        const size_t vo = (size_t)(lo + c) * ld + i;
        dot2_acc(make_float2(Uh[vo], 0.f), make_float2(Ul[vo], 0.f), wh, wl, S[c], C[c]);
      }
    dot2_acc(wh, wl, wh, wl, S[KW], C[KW]);
  }
  ff v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = dot2_value(S[k], C[k]);
  block_sum<true, K>(v, sh, tot);
  const int G = gridDim.x;
  if (threadIdx.x < K) part[(size_t)threadIdx.x * G + blockIdx.x] = tot[threadIdx.x];
  griddep_launch();
}

template <int KW>
__global__ void __launch_bounds__(NT) k_iom_update_ff(KState* ks, ff* part, Basis U, int j, size_t n_aug, int Gd) {
  __shared__ float2 cf[KW];
  __shared__ IomScalars sc;
  __shared__ ff sh[NW];
  __shared__ ff tot[1];
  const int lo = max(0, j - KW + 1), nwin = j - lo + 1;
  const size_t ld = U.ld, ng = n_aug / 4;
  float* __restrict__ Uh = U.h;
  float* __restrict__ Ul = U.l;
  const size_t tid = blockIdx.x * (size_t)NT + threadIdx.x, nthr = (size_t)gridDim.x * NT;
  // the first trip's vectors (w' and the window slots: see above) before
  // the wait; the window products' partials (the predecessor's) after it
  float4 pwh = make_float4(0.f, 0.f, 0.f, 0.f), pwl = pwh, pxh[KW], pxl[KW];
  if (tid < ng) {
    pwh = *reinterpret_cast<const float4*>(Uh + (j + 1) * ld + 4 * tid);
    pwl = *reinterpret_cast<const float4*>(Ul + (j + 1) * ld + 4 * tid);
#pragma unroll
    for (int c = 0; c < KW; ++c) {
      const size_t vo = (size_t)(lo + (c < nwin ? c : 0)) * ld + 4 * tid;
      pxh[c] = __ldg(reinterpret_cast<const float4*>(Uh + vo));
      pxl[c] = __ldg(reinterpret_cast<const float4*>(Ul + vo));
    }
  }
  griddep_wait();
  const int go = iom_prologue_ff(ks, part, j, lo, nwin, KW + 1, Gd, gridDim.x, cf, &sc);
  if (go <= 0) {
    if (go == 0) write_iom_scalars(ks, sc, j, lo, nwin);  // a breakdown at j: record it
    return;
  }
  const float2 cjh = make_float2(sc.cj.h, sc.cj.h), cjl = make_float2(sc.cj.l, sc.cj.l);
  float2 S = make_float2(0.f, 0.f), C = make_float2(0.f, 0.f);
  for (size_t g = tid; g < ng; g += nthr) {
    const size_t o = 4 * g;
    float4 wh = pwh, wl = pwl, xh[KW], xl[KW];
    if (g == tid) {
#pragma unroll
      for (int c = 0; c < KW; ++c) xh[c] = pxh[c], xl[c] = pxl[c];
    } else {
      wh = *reinterpret_cast<const float4*>(Uh + (j + 1) * ld + o);
      wl = *reinterpret_cast<const float4*>(Ul + (j + 1) * ld + o);
#pragma unroll
      for (int c = 0; c < KW; ++c) {
        const size_t vo = (size_t)(lo + (c < nwin ? c : 0)) * ld + o;
        xh[c] = __ldg(reinterpret_cast<const float4*>(Uh + vo));
        xl[c] = __ldg(reinterpret_cast<const float4*>(Ul + vo));
      }
    }
    float2 uh0 = lo2(wh), uh1 = hi2(wh), ul0 = lo2(wl), ul1 = hi2(wl);
    ff2_scale(uh0, ul0, cjh, cjl);  // w = c_j w'
    ff2_scale(uh1, ul1, cjh, cjl);
#pragma unroll
    for (int c = 0; c < KW; ++c)
      if (c < nwin) {
        const float2 ah = make_float2(cf[c].x, cf[c].x), al = make_float2(cf[c].y, cf[c].y);
        axpy2_acc(ah, al, lo2(xh[c]), lo2(xl[c]), uh0, ul0);
        axpy2_acc(ah, al, hi2(xh[c]), hi2(xl[c]), uh1, ul1);
      }
    ff2_norm(uh0, ul0);
    ff2_norm(uh1, ul1);
    *reinterpret_cast<float4*>(Uh + (j + 1) * ld + o) = make_float4(uh0.x, uh0.y, uh1.x, uh1.y);
    *reinterpret_cast<float4*>(Ul + (j + 1) * ld + o) = make_float4(ul0.x, ul0.y, ul1.x, ul1.y);
    dot2_acc(uh0, ul0, uh0, ul0, S, C);
    dot2_acc(uh1, ul1, uh1, ul1, S, C);
  }
  for (size_t i = 4 * ng + tid; i < n_aug; i += nthr) {  // ragged end
    ff x = ff_mul(ff{sc.cj.h, sc.cj.l}, ff{Uh[(j + 1) * ld + i], Ul[(j + 1) * ld + i]});
    for (int c = 0; c < nwin; ++c) {
      const size_t vo = (size_t)(lo + c) * ld + i;
      x = ff_fma(ff{cf[c].x, cf[c].y}, ff{Uh[vo], Ul[vo]}, x);
    }
    Uh[(j + 1) * ld + i] = x.h;
    Ul[(j + 1) * ld + i] = x.l;
    dot2_acc(make_float2(x.h, 0.f), make_float2(x.l, 0.f), make_float2(x.h, 0.f), make_float2(x.l, 0.f), S, C);
  }
  ff v[1] = {dot2_value(S, C)};
  block_sum<true, 1>(v, sh, tot);
  if (threadIdx.x == 0) part[IOM_UPD_OFF + (j & 1) * RB_MAX + blockIdx.x] = tot[0];
  griddep_launch();
  write_iom_scalars(ks, sc, j, lo, nwin);
}

// FP64 form: four elements per thread per trip, loads first.
template <int KW>
__global__ void __launch_bounds__(NT) k_iom_dots(KState* ks, double* part, Basis U, int j, size_t n_aug) {
  griddep_wait();
  constexpr int K = KW + 1;
  __shared__ double sh[NW * K];
  __shared__ double tot[K];
  const int lo = max(0, j - KW + 1), nwin = j - lo + 1;
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  const size_t ng = n_aug / 4;
  const size_t tid = blockIdx.x * (size_t)NT + threadIdx.x, nthr = (size_t)gridDim.x * NT;
  for (size_t g = tid; g < ng; g += nthr) {
    const Quad<false> w = ldq<false>(U, j + 1, g);
    Quad<false> x[KW];
#pragma unroll
    for (int c = 0; c < KW; ++c) x[c] = ldq<false>(U, lo + (c < nwin ? c : 0), g);
#pragma unroll
    for (int c = 0; c < KW; ++c)
      if (c < nwin)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[c] = fma(x[c].v[e], w.v[e], acc[c]);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[KW] = fma(w.v[e], w.v[e], acc[KW]);
  }
  for (size_t i = 4 * ng + tid; i < n_aug; i += nthr) {
    const double wi = ldb<false>(U, j + 1, i);
#pragma unroll
    for (int c = 0; c < KW; ++c)
      if (c < nwin) acc[c] = fma(ldb<false>(U, lo + c, i), wi, acc[c]);
    acc[KW] = fma(wi, wi, acc[KW]);
  }
  block_sum<false, K>(acc, sh, tot);
  const int G = gridDim.x;
  if (threadIdx.x < K) part[(size_t)threadIdx.x * G + blockIdx.x] = tot[threadIdx.x];
  griddep_launch();
}

template <int KW>
__global__ void __launch_bounds__(NT) k_iom_update(KState* ks, double* part, Basis U, int j, size_t n_aug, int Gd) {
  griddep_wait();
  __shared__ double cf[IOP_MAX];
  __shared__ double sh[NW];
  __shared__ double tot[1];
  const int lo = max(0, j - KW + 1), nwin = j - lo + 1;
  __shared__ double cj;
  if (!iom_prologue<false>(ks, part, j, lo, nwin, KW + 1, Gd, gridDim.x, cf, &cj)) return;
  double nrm[1] = {0.0};
  const size_t ng = n_aug / 4;
  const size_t tid = blockIdx.x * (size_t)NT + threadIdx.x, nthr = (size_t)gridDim.x * NT;
  for (size_t g = tid; g < ng; g += nthr) {
    Quad<false> w = ldq<false>(U, j + 1, g);
    Quad<false> x[KW];
#pragma unroll
    for (int c = 0; c < KW; ++c) x[c] = ldq<false>(U, lo + (c < nwin ? c : 0), g);
#pragma unroll
    for (int e = 0; e < 4; ++e) w.v[e] *= cj;  // w = c_j w'
#pragma unroll
    for (int c = 0; c < KW; ++c)
      if (c < nwin)
#pragma unroll
        for (int e = 0; e < 4; ++e) w.v[e] = fma(cf[c], x[c].v[e], w.v[e]);
#pragma unroll
    for (int e = 0; e < 4; ++e) nrm[0] = fma(w.v[e], w.v[e], nrm[0]);
    stq<false>(U, j + 1, g, w);
  }
  for (size_t i = 4 * ng + tid; i < n_aug; i += nthr) {
    double w = cj * ldb<false>(U, j + 1, i);
    for (int c = 0; c < nwin; ++c) w = fma(cf[c], ldb<false>(U, lo + c, i), w);
    stb<false>(U, j + 1, i, w);
    nrm[0] = fma(w, w, nrm[0]);
  }
  block_sum<false, 1>(nrm, sh, tot);
  if (threadIdx.x == 0) part[IOM_UPD_OFF + (j & 1) * RB_MAX + blockIdx.x] = tot[0];
  griddep_launch();
}

// ---- mixed form: FP32 operator applies on an FP64 Krylov basis ----
// Slot i keeps its FP64 entries in U.d and their FP32 rounding in the shadow
// plane U.h, which the FP32 operator apply reads.  The operator apply of step
// j writes the top N entries of w' = A_hat slot_j in FP32 to the shadow plane
// of slot j+1 (the FP32 operator's result, exact there) and the P tail
// entries in FP64 to slot j+1.  The window-products launch widens w' exactly
// (cvt.cuh, integer pipes) and forms the inner products in FP64; the update
// writes slot j+1 in FP64 and its FP32 rounding to the shadow plane.  |w'|^2
// only scales the happy-breakdown test: its top part is summed in FP32 (one
// FP64 operation fewer per element on the narrow FP64 pipe; the true-scale
// slots keep w' within a few orders of magnitude of the operator's norm).
// ||slot_{j+1}||^2 likewise, from the FP32 rounding the update writes
// (compensated FP32 sums per thread, FP64 across threads): it sets
// c_{j+1} = 1 / ||slot_{j+1}|| and H(j+1, j) = ||slot_{j+1}|| together, so
// H(j+1, j) v_{j+1} = slot_{j+1} and the Arnoldi relation hold whatever its
// rounding; only the unit length of v_{j+1} depends on it (to about 1e-7),
// and the update's FP64 operations are the window's alone.
// The update scales w' by c_j in FP32 too (part of the operator apply on the
// unit vector v_j), so its FP64 operations are the window's and the norm's.
// Loads before griddepcontrol.wait as in the float-float kernels above.

// Entry i of w' (slot j1): FP32 top part widened, FP64 tail.
__device__ __forceinline__ double mx_w(const Basis& U, int j1, size_t i, size_t N) {
  const size_t o = (size_t)j1 * U.ld + i;
  return i < N ? f32_to_f64_exact(U.h[o]) : U.d[o];
}

template <int KW>
__global__ void __launch_bounds__(NT) k_iom_dots_mx(KState* ks, double* part, Basis U, int j, size_t N,
                                                    size_t n_aug) {
  constexpr int K = KW + 1;
  __shared__ double sh[K * NT];
  __shared__ double tot[K];
  const int lo = max(0, j - KW + 1), nwin = j - lo + 1;
  double acc[KW], acc2[KW];  // two chains a slot (more FP64 operations in flight)
#pragma unroll
  for (int c = 0; c < KW; ++c) acc[c] = acc2[c] = 0.0;
  float wn = 0.0f;     // |w'|^2 of the top part (FP32)
  double wnt = 0.0;    // and of the ragged end and tail
  const size_t ld = U.ld, ng = N / 4;
  const size_t tid = blockIdx.x * (size_t)NT + threadIdx.x, nthr = (size_t)gridDim.x * NT;
  // the first trip's window slots before the wait (written by the previous update)
  Quad<false> px[KW];
  if (tid < ng)
#pragma unroll
    for (int c = 0; c < KW; ++c) px[c] = ldq<false>(U, lo + (c < nwin ? c : 0), tid);
  griddep_wait();
  const float* __restrict__ wtop = U.h + (size_t)(j + 1) * ld;
  // quad g's products from its loaded inputs
  auto body = [&](const float4 wf, const Quad<false>* x) {
    const double w[4] = {f32_to_f64_exact(wf.x), f32_to_f64_exact(wf.y), f32_to_f64_exact(wf.z),
                         f32_to_f64_exact(wf.w)};
#pragma unroll
    for (int c = 0; c < KW; ++c)
      if (c < nwin) {
        acc[c] = fma(x[c].v[1], w[1], fma(x[c].v[0], w[0], acc[c]));
        acc2[c] = fma(x[c].v[3], w[3], fma(x[c].v[2], w[2], acc2[c]));
      }
    wn = fmaf(wf.x, wf.x, fmaf(wf.y, wf.y, fmaf(wf.z, wf.z, fmaf(wf.w, wf.w, wn))));
  };
  auto load = [&](size_t g, float4& wf, Quad<false>* x) {
    wf = __ldg(reinterpret_cast<const float4*>(wtop + 4 * g));
#pragma unroll
    for (int c = 0; c < KW; ++c) x[c] = ldq<false>(U, lo + (c < nwin ? c : 0), g);
  };
  size_t g = tid;
  if (g < ng) {  // the first trip (its slots loaded before the wait)
    body(__ldg(reinterpret_cast<const float4*>(wtop + 4 * g)), px);
    g += nthr;
  }
  if constexpr (KW <= 2) {  // short windows: two trips' loads in flight at once
    for (; g + nthr < ng; g += 2 * nthr) {
      float4 wa, wb;
      Quad<false> xa[KW], xb[KW];
      load(g, wa, xa);
      load(g + nthr, wb, xb);
      body(wa, xa);
      body(wb, xb);
    }
  }
  for (; g < ng; g += nthr) {
    float4 wa;
    Quad<false> xa[KW];
    load(g, wa, xa);
    body(wa, xa);
  }
#pragma unroll
  for (int c = 0; c < KW; ++c) acc[c] += acc2[c];
  for (size_t i = 4 * ng + tid; i < n_aug; i += nthr) {  // ragged end and the augmentation tail
    const double wi = mx_w(U, j + 1, i, N);
#pragma unroll
    for (int c = 0; c < KW; ++c)
      if (c < nwin) acc[c] = fma(ldb<false>(U, lo + c, i), wi, acc[c]);
    wnt = fma(wi, wi, wnt);
  }
  double v[K];
#pragma unroll
  for (int c = 0; c < KW; ++c) v[c] = acc[c];
  v[KW] = (double)wn + wnt;
  block_sum_1w<K>(v, sh, tot);
  const int G = gridDim.x;
  if (threadIdx.x < K) part[(size_t)threadIdx.x * G + blockIdx.x] = tot[threadIdx.x];
  griddep_launch();
}

template <int KW>
__global__ void __launch_bounds__(NT) k_iom_update_mx(KState* ks, double* part, Basis U, int j, size_t N,
                                                      size_t n_aug, int Gd) {
  __shared__ double cf[IOP_MAX];
  __shared__ double sh[NT];
  __shared__ double tot[1];
  __shared__ double cj;
  const int lo = max(0, j - KW + 1), nwin = j - lo + 1;
  const size_t ld = U.ld, ng = N / 4;
  const size_t tid = blockIdx.x * (size_t)NT + threadIdx.x, nthr = (size_t)gridDim.x * NT;
  float* __restrict__ Uh = U.h;
  // the first trip's w' and window slots before the wait (written by the
  // operator apply and the previous update); the window products' partials after it
  float4 pwf = make_float4(0.f, 0.f, 0.f, 0.f);
  Quad<false> px[KW];
  if (tid < ng) {
    pwf = *reinterpret_cast<const float4*>(Uh + (size_t)(j + 1) * ld + 4 * tid);
#pragma unroll
    for (int c = 0; c < KW; ++c) px[c] = ldq<false>(U, lo + (c < nwin ? c : 0), tid);
  }
  griddep_wait();
  if (!iom_prologue<false>(ks, part, j, lo, nwin, KW + 1, Gd, gridDim.x, cf, &cj)) return;
  const double c_j = cj;
  // c_j w' = A_hat v_j: the operator's FP32 output scaled to the unit basis
  // vector in FP32 (one rounding, at the level of the FP32 operator's own),
  // then widened exactly; the slots stay at true scale
  const float c_jf = f64_to_f32_rn(c_j);
  double nrm[1] = {0.0};
  float ns = 0.0f, nc = 0.0f;  // |slot_{j+1}|^2 of the top part from its FP32 rounding (compensated sum)
  // quad g from its loaded inputs: the update, both stores, the norm term
  auto finish = [&](size_t g, const float4 wf, const Quad<false>* x) {
    Quad<false> w;
    w.v[0] = f32_to_f64_exact(__fmul_rn(c_jf, wf.x));
    w.v[1] = f32_to_f64_exact(__fmul_rn(c_jf, wf.y));
    w.v[2] = f32_to_f64_exact(__fmul_rn(c_jf, wf.z));
    w.v[3] = f32_to_f64_exact(__fmul_rn(c_jf, wf.w));
#pragma unroll
    for (int c = 0; c < KW; ++c)
      if (c < nwin)
#pragma unroll
        for (int e = 0; e < 4; ++e) w.v[e] = fma(cf[c], x[c].v[e], w.v[e]);
    stq<false>(U, j + 1, g, w);
    const float4 sh =
        make_float4(f64_to_f32_rn(w.v[0]), f64_to_f32_rn(w.v[1]), f64_to_f32_rn(w.v[2]), f64_to_f32_rn(w.v[3]));
    *reinterpret_cast<float4*>(Uh + (size_t)(j + 1) * ld + 4 * g) = sh;
    const float sq = __fmaf_rn(sh.x, sh.x, __fmaf_rn(sh.y, sh.y, __fmaf_rn(sh.z, sh.z, __fmul_rn(sh.w, sh.w))));
    const float y = __fsub_rn(sq, nc), t = __fadd_rn(ns, y);  // Kahan's compensated summation
    nc = __fsub_rn(__fsub_rn(t, ns), y);
    ns = t;
  };
  auto load = [&](size_t g, float4& wf, Quad<false>* x) {
    wf = *reinterpret_cast<const float4*>(Uh + (size_t)(j + 1) * ld + 4 * g);
#pragma unroll
    for (int c = 0; c < KW; ++c) x[c] = ldq<false>(U, lo + (c < nwin ? c : 0), g);
  };
  size_t g = tid;
  if (g < ng) {  // the first trip, loaded before the wait
    finish(g, pwf, px);
    g += nthr;
  }
  for (; g + nthr < ng; g += 2 * nthr) {  // two trips' loads in flight at once
    float4 wa, wb;
    Quad<false> xa[KW], xb[KW];
    load(g, wa, xa);
    load(g + nthr, wb, xb);
    finish(g, wa, xa);
    finish(g + nthr, wb, xb);
  }
  if (g < ng) {
    float4 wa;
    Quad<false> xa[KW];
    load(g, wa, xa);
    finish(g, wa, xa);
  }
  nrm[0] = f32_to_f64_exact(ns) - f32_to_f64_exact(nc);
  for (size_t i = 4 * ng + tid; i < n_aug; i += nthr) {  // ragged end (FP32 scaling) and the FP64 tail
    double w = (i < N) ? f32_to_f64_exact(__fmul_rn(c_jf, Uh[(size_t)(j + 1) * ld + i])) : c_j * U.d[(size_t)(j + 1) * ld + i];
    for (int c = 0; c < nwin; ++c) w = fma(cf[c], ldb<false>(U, lo + c, i), w);
    stb<false>(U, j + 1, i, w);
    if (i < N) Uh[(size_t)(j + 1) * ld + i] = f64_to_f32_rn(w);
    nrm[0] = fma(w, w, nrm[0]);
  }
  block_sum_1w<1>(nrm, sh, tot);
  if (threadIdx.x == 0) part[IOM_UPD_OFF + (j & 1) * RB_MAX + blockIdx.x] = tot[0];
  griddep_launch();
}

// Dense exponential of the m x m leading block of H: scaling and squaring,
// exp(H) = T(H / 2^s)^(2^s) with ||H / 2^s||_1 <= 1/2 and T the degree-18
// Taylor polynomial, evaluated by Paterson-Stockmeyer in X^4:
//   T(X) = B_0 + X^4 (B_1 + X^4 (B_2 + X^4 (B_3 + X^4 B_4))),
//   B_j = sum_{i<4} X^i / (4j+i)!,  B_4 = I/16! + X/17! + X^2/18!,
// i.e. 3 products for X^2, X^3, X^4 and 4 Horner products instead of 18.
// On a cluster of PHI_CL CTAs: every CTA keeps full copies of the matrices in
// shared memory; each product is split by rows across the CTAs, each entry's
// sum over k across PHI_KS adjacent lanes (shorter dependent chains), and
// every CTA writes its rows into all CTAs' copies (distributed shared
// memory), followed by one cluster barrier.  Results alternate between two
// buffers, so a CTA never overwrites a copy another CTA may still read.
// The arithmetic is FP64 (FP64 form) or float-float on the FP32 pipes (mixed
// form: 48-bit significands, far below its tolerances; GB300's FP64 pipe
// runs about 2 FMA per SM per clock).
constexpr int PHI_CL = 8;
constexpr int PHI_NT = 256;
constexpr int PHI_KS = 4;
// Largest m whose pair (H_{m-1} and H_m, six copies each) fits the 227 KB of
// shared memory a CTA may have.
constexpr int PHI_PAIR_MAX = 49;
static_assert(6 * 8 * (PHI_PAIR_MAX * PHI_PAIR_MAX + (PHI_PAIR_MAX - 1) * (PHI_PAIR_MAX - 1)) + 256 <= 227 * 1024,
              "the pair fits one CTA's shared memory");

// 1/k!, k = 0..18, as FP64 and as float-float pairs (computed on the host).
struct PhiConst {
  double d[19];
  float2 f[19];
};

template <typename T>
struct PhiT;
template <>
struct PhiT<double> {
  using S = double;  // scalar type of norms and power-of-two scales
  __device__ static double zero() { return 0.0; }
  __device__ static double cnst(const PhiConst& c, int k) { return c.d[k]; }
  __device__ static double mad(double a, double b, double c) { return fma(a, b, c); }
  __device__ static double add(double a, double b) { return a + b; }
  __device__ static double pow2(double a, double s) { return a * s; }
  __device__ static double from_d(double x) { return x; }
  __device__ static double to_d(double x) { return x; }
  __device__ static double mag(double x) { return fabs(x); }
  __device__ static double shfl_xor(double x, int m) { return __shfl_xor_sync(0xffffffffu, x, m); }
};
template <>
struct PhiT<ff> {
  using S = float;
  __device__ static ff zero() { return ff{0.0f, 0.0f}; }
  __device__ static ff cnst(const PhiConst& c, int k) { return ff{c.f[k].x, c.f[k].y}; }
  __device__ static ff mad(ff a, ff b, ff c) { return ff_fma(a, b, c); }
  __device__ static ff add(ff a, ff b) { return ff_add(a, b); }
  __device__ static ff pow2(ff a, float s) { return ff{a.h * s, a.l * s}; }
  __device__ static ff from_d(double x) { return ff_from_double(x); }
  __device__ static double to_d(ff x) { return ff_to_double(x); }
  __device__ static float mag(ff x) { return fabsf(x.h); }
  __device__ static ff shfl_xor(ff x, int m) {
    return ff{__shfl_xor_sync(0xffffffffu, x.h, m), __shfl_xor_sync(0xffffffffu, x.l, m)};
  }
};

// The matrices of one evaluation: nb (1 or 2) square diagonal blocks stored
// packed, block 0 n0 x n0 row-major from offset 0, block 1 n1 x n1 from off1,
// tot entries in all.  With two blocks exp(H_{m-1}) and exp(H_m) are formed
// together (the change of the approximation since m - 1 for the float-float
// form's test).
struct PhiBlocks {
  int nb, n0, n1, off1, tot;
  __device__ int n(int b) const { return b ? n1 : n0; }
  __device__ int off(int b) const { return b ? off1 : 0; }
  __device__ void rc(int idx, int& b, int& r, int& c) const {
    b = (nb > 1 && idx >= off1) ? 1 : 0;
    const int o = idx - off(b), nn = n(b);
    r = o / nn;
    c = o - r * nn;
  }
};

// C = A B blockwise within the group of PHI_CL CTAs from cluster rank base
// (which all hold the same matrices).  The entries are split evenly across
// the group's CTAs, each entry's sum over k across PHI_KS adjacent lanes;
// every CTA writes its entries into all the group's copies, then one
// barrier of the whole cluster.
template <typename T>
__device__ void cl_matmul(cg::cluster_group& cl, const T* A, const T* B, T* C, const PhiBlocks& bk, int base) {
  using PT = PhiT<T>;
  const int rank = (int)cl.block_rank() - base;
  const int e0 = (bk.tot * rank) / PHI_CL, e1 = (bk.tot * (rank + 1)) / PHI_CL;
  T* dst[PHI_CL];
#pragma unroll
  for (int t = 0; t < PHI_CL; ++t) dst[t] = cl.map_shared_rank(C, base + t);
  const int nout = e1 - e0;
  const int rounds = (nout * PHI_KS + blockDim.x - 1) / blockDim.x;  // the same for every thread
  for (int rd = 0; rd < rounds; ++rd) {
    const int g = rd * blockDim.x + threadIdx.x;
    const int o = g / PHI_KS, q = g - o * PHI_KS;  // entry e0 + o, part q of its sum
    const int idx = e0 + o;
    T acc = PT::zero();
    if (o < nout) {
      int b, r, c;
      bk.rc(idx, b, r, c);
      const int n = bk.n(b);
      const T* Ab = A + bk.off(b) + r * n;
      const T* Bb = B + bk.off(b) + c;
      for (int k = q; k < n; k += PHI_KS) acc = PT::mad(Ab[k], Bb[k * n], acc);
    }
#pragma unroll
    for (int off = 1; off < PHI_KS; off <<= 1) acc = PT::add(acc, PT::shfl_xor(acc, off));
    if (o < nout && q == 0) {
#pragma unroll
      for (int t = 0; t < PHI_CL; ++t) dst[t][idx] = acc;
    }
  }
  cl.sync();
}

// GROUPS = 1: one cluster of PHI_CL CTAs (pair: H_{m-1} and H_m packed
// together).  GROUPS = 2: a cluster of 2 PHI_CL CTAs, the first group
// evaluating H_{m-1}, the second H_m, each at a single matrix's cost; the
// second group's first CTA reads y_{m-1} from the first group's shared memory.
// Launched with the cluster size as a launch attribute.
template <typename T, int GROUPS>
__global__ void __launch_bounds__(PHI_NT)
k_phi(KState* ks, int m_req, double beta, double tol, int force, int diff_rule, const void* iom_part, int iom_kf,
      int iom_gu, int pair, const PhiConst pc) {
  const bool iom_ff = iom_kf == KF_FF;
  using PT = PhiT<T>;
  using SC = typename PT::S;
  cg::cluster_group cl = cg::this_cluster();
  if (beta < 0.0) beta = ks->beta;  // computed on the device by the norms kernel
  extern __shared__ __align__(16) unsigned char phi_smem[];
  __shared__ int s_m;
  __shared__ SC s_norm;
  __shared__ double s_hm;  // h_{m,m-1}
  __shared__ int s_brk;
  if (threadIdx.x == 0) {
    const int b = ks->breakdown_at;
    s_m = (b > 0 && b < m_req) ? b : m_req;
    s_brk = (b > 0 && b <= m_req) ? 1 : 0;
    s_hm = ks->H[(s_m - 1) * (MMAX + 1) + s_m];
  }
  __syncthreads();
  // Incomplete orthogonalisation: h_{m,m-1} = ||slot_m|| from the partials of
  // the last update launch (every CTA sums them alike).
  if (iom_part != nullptr && s_m == m_req && !s_brk) {
    const int off = IOM_UPD_OFF + (((m_req - 1) & 1) ? RB_MAX : 0);
    if (threadIdx.x < 32) {
      double x = 0.0;
      if (iom_ff) {
        ff t{0.0f, 0.0f};
        for (int g = threadIdx.x; g < iom_gu; g += 32) t = ff_add(t, static_cast<const ff*>(iom_part)[off + g]);
        for (int o = 16; o > 0; o >>= 1) t = ff_add(t, ff_shfl_down(t, o));
        x = ff_to_double(t);
      } else {
        for (int g = threadIdx.x; g < iom_gu; g += 32) x += static_cast<const double*>(iom_part)[off + g];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      }
      if (threadIdx.x == 0) {
        const double ns = sqrt(x);
        const bool brk = ns <= 1e-13 * ks->wnp[(m_req - 1) & 1] || ns == 0.0;
        s_hm = ns;
        s_brk = brk ? 1 : 0;
        if (cl.block_rank() == 0) {
          ks->H[(m_req - 1) * (MMAX + 1) + m_req] = s_hm;
          if (brk && ks->breakdown_at == 0) ks->breakdown_at = m_req;
        }
      }
    }
    __syncthreads();
  }
  const int m = s_m;
  const int grp = (GROUPS == 2) ? (int)cl.block_rank() / PHI_CL : 0, base = grp * PHI_CL;
  const int lead = (GROUPS == 2) ? PHI_CL : 0;  // the CTA that forms the decision
  // pair (one group): H_{m-1} as block 0 beside H_m (block 1), the same
  // scaling for both (the leading block's 1-norm is at most H_m's).  Two
  // groups: this group's matrix alone, in buffers of m x m entries in both
  // groups (the same offsets, for the remote read of y_{m-1}).
  const bool two = (GROUPS == 1) && pair && m >= 2 && !s_brk;
  const int mg = (GROUPS == 2 && grp == 0) ? m - 1 : m;
  PhiBlocks bk;
  bk.nb = two ? 2 : 1;
  bk.n0 = two ? m - 1 : mg;
  bk.n1 = m;
  bk.off1 = two ? (m - 1) * (m - 1) : 0;
  bk.tot = two ? bk.off1 + m * m : mg * mg;
  const int tot = bk.tot, ncol = bk.n0 + (two ? m : 0);
  const int stride = (GROUPS == 2) ? m * m : tot;
  T* X = reinterpret_cast<T*>(phi_smem);
  T* X2 = X + stride;
  T* X3 = X2 + stride;
  T* X4 = X3 + stride;
  T* T0 = X4 + stride;
  T* T1 = T0 + stride;
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    int b, r, c;
    bk.rc(idx, b, r, c);
    X[idx] = PT::from_d(ks->H[c * (MMAX + 1) + r]);
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // largest column sum over both blocks (two groups: of H_m, in every CTA alike)
    SC mx = 0;
    if (GROUPS == 2) {
      for (int c = threadIdx.x; c < m; c += 32) {
        SC cs = 0;
        for (int r = 0; r < m; ++r) cs += PT::mag(PT::from_d(ks->H[c * (MMAX + 1) + r]));
        mx = cs > mx ? cs : mx;
      }
    } else {
      for (int cc = threadIdx.x; cc < ncol; cc += 32) {
        const int b = (cc >= bk.n0) ? 1 : 0, c = cc - (b ? bk.n0 : 0), n = bk.n(b);
        const T* Xb = X + bk.off(b);
        SC cs = 0;
        for (int r = 0; r < n; ++r) cs += PT::mag(Xb[r * n + c]);
        mx = cs > mx ? cs : mx;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const SC o = __shfl_down_sync(0xffffffffu, mx, off);
      mx = o > mx ? o : mx;
    }
    if (threadIdx.x == 0) s_norm = mx;
  }
  __syncthreads();
  int sq = 0;
  if (s_norm > SC(0.5)) sq = (int)ceil(log2(s_norm / SC(0.5)));
  const SC scale = (SC)ldexp(1.0f, -sq);  // a power of two: exact in both types
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) X[idx] = PT::pow2(X[idx], scale);
  cl.sync();  // every CTA has its scaled copy before any remote write lands
  cl_matmul(cl, X, X, X2, bk, base);
  cl_matmul(cl, X2, X, X3, bk, base);
  cl_matmul(cl, X2, X2, X4, bk, base);
  // E = B_4
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    int b, r, c;
    bk.rc(idx, b, r, c);
    const T diag = (r == c) ? PT::cnst(pc, 16) : PT::zero();
    T0[idx] = PT::mad(PT::cnst(pc, 18), X2[idx], PT::mad(PT::cnst(pc, 17), X[idx], diag));
  }
  __syncthreads();
  T* E = T0;
  T* F = T1;
  for (int j = 3; j >= 0; --j) {
    cl_matmul(cl, X4, E, F, bk, base);
    const T c0 = PT::cnst(pc, 4 * j), c1 = PT::cnst(pc, 4 * j + 1), c2 = PT::cnst(pc, 4 * j + 2),
            c3 = PT::cnst(pc, 4 * j + 3);
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
      int b, r, c;
      bk.rc(idx, b, r, c);
      const T f = (r == c) ? PT::add(F[idx], c0) : F[idx];
      F[idx] = PT::mad(c3, X3[idx], PT::mad(c2, X2[idx], PT::mad(c1, X[idx], f)));
    }
    __syncthreads();
    T* t = E;
    E = F;
    F = t;
  }
  for (int k = 0; k < sq; ++k) {
    cl_matmul(cl, E, E, F, bk, base);
    T* t = E;
    E = F;
    F = t;
  }
  if ((int)cl.block_rank() == lead) {
    __shared__ double s_d2[PHI_NT / 32];
    // y = exp(H_m) e_1: column 0 of the last block
    const T* Em = E + bk.off1;
    // y_{m-1}: column 0 of block 0 (pair), or of the first group's matrix
    const bool paired = two || GROUPS == 2;
    const T* Ep = (GROUPS == 2) ? cl.map_shared_rank(E, 0) : E;
    // squared change of y since m - 1 (pair) or since the previous check
    // (entries beyond the shorter vector count fully)
    double d2 = 0.0;
    const int mp = paired ? m - 1 : ks->mprev;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const double yo = (i < mp) ? (paired ? PT::to_d(Ep[i * (m - 1)]) : ks->yprev[i]) : 0.0;
      const double di = PT::to_d(Em[i * m]) - yo;
      d2 += di * di;
    }
    for (int off = 16; off > 0; off >>= 1) d2 += __shfl_down_sync(0xffffffffu, d2, off);
    if ((threadIdx.x & 31) == 0) s_d2[threadIdx.x >> 5] = d2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double dsum = 0.0;
      for (int w = 0; w < PHI_NT / 32; ++w) dsum += s_d2[w];
      const bool brk = s_brk != 0;
      const double hm = s_hm;
      const double err = brk ? 0.0 : beta * hm * fabs(PT::to_d(Em[(m - 1) * m]));
      const double dif = (mp > 0) ? beta * sqrt(dsum) : 1.0 / 0.0;
      const bool ok = brk || err <= tol * beta || (diff_rule && dif <= tol * beta);
      ks->err = diff_rule ? fmin(err, dif) : err;
      ks->accept = (force || ok) ? 1 : 0;
      ks->m_eff = m;
      ks->norm1 = (double)s_norm;
      ks->squarings = sq;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const double y = PT::to_d(Em[i * m]);
      ks->ycoef[i] = beta * y * ks->vscale[i];
      ks->yprev[i] = y;
    }
    if (threadIdx.x == 0) ks->mprev = m;
  }
  cl.sync();  // no CTA exits while others may still write into its shared memory
}

template <bool FF>
__global__ void __launch_bounds__(NT) k_combine(const KState* ks, Basis U, Vec base, Vec out, size_t N,
                                                int if_accepted) {
  if (if_accepted && ks->accept == 0) return;
  using A = Acc<FF>;
  __shared__ typename A::T cf[MMAX + 1];
  const int m = ks->m_eff;
  for (int i = threadIdx.x; i < m; i += NT) cf[i] = from_d<FF>(ks->ycoef[i]);
  __syncthreads();
  const bool base_d = base.d != nullptr, base_ff = base.h != nullptr;
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < N; i += (size_t)gridDim.x * NT) {
    typename A::T x = A::zero();
    for (int k = 0; k < m; ++k) x = fma_acc<FF>(cf[k], ldb<FF>(U, k, i), x);
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

// Float-float combination: x = sum_{k < m} ycoef_k slot_k for a quad of
// elements per thread (two float4 loads per vector, the next vector's loads
// issued before this one's arithmetic; packed compensated accumulation), then
// out = base + x, out FP64 (d) or float-float (h, l), base FP64, float-float or
// absent.
__global__ void __launch_bounds__(NT) k_combine_ff(const KState* ks, Basis U, Vec base, Vec out, size_t N,
                                                   int if_accepted) {
  if (if_accepted && ks->accept == 0) return;
  __shared__ float2 cf[MMAX + 1];
  const int m = ks->m_eff;
  for (int i = threadIdx.x; i < m; i += NT) {
    const ff c = ff_from_double(ks->ycoef[i]);
    cf[i] = make_float2(c.h, c.l);
  }
  __syncthreads();
  const size_t ld = U.ld, ng = N / 4;
  const float* __restrict__ Uh = U.h;
  const float* __restrict__ Ul = U.l;
  const bool base_d = base.d != nullptr, base_ff = base.h != nullptr;
  auto emit = [&](size_t i, ff x) {
    if (out.d != nullptr) {
      double o = ff_to_double(x);
      if (base_d) o += base.d[i];
      if (base_ff) o += ff_to_double(ff{base.h[i], base.l[i]});
      out.d[i] = o;
    } else {
      if (base_ff) x = ff_add(x, ff{base.h[i], base.l[i]});
      if (base_d) x = ff_add(x, ff_from_double(base.d[i]));
      out.h[i] = x.h;
      out.l[i] = x.l;
    }
  };
  const float2 z2 = make_float2(0.f, 0.f);
  const size_t tid = blockIdx.x * (size_t)NT + threadIdx.x, nthr = (size_t)gridDim.x * NT;
  for (size_t g = tid; g < ng; g += nthr) {
    const size_t o = 4 * g;
    float2 xh0 = z2, xh1 = z2, xl0 = z2, xl1 = z2;
    float4 nh = make_float4(0.f, 0.f, 0.f, 0.f), nl = nh;
    if (m > 0) {
      nh = __ldg(reinterpret_cast<const float4*>(Uh + o));
      nl = __ldg(reinterpret_cast<const float4*>(Ul + o));
    }
    for (int k = 0; k < m; ++k) {
      const float4 bh = nh, bl = nl;
      if (k + 1 < m) {
        nh = __ldg(reinterpret_cast<const float4*>(Uh + (size_t)(k + 1) * ld + o));
        nl = __ldg(reinterpret_cast<const float4*>(Ul + (size_t)(k + 1) * ld + o));
      }
      const float2 ah = make_float2(cf[k].x, cf[k].x), al = make_float2(cf[k].y, cf[k].y);
      axpy2_acc(ah, al, lo2(bh), lo2(bl), xh0, xl0);
      axpy2_acc(ah, al, hi2(bh), hi2(bl), xh1, xl1);
      if ((k & 15) == 15) {
        ff2_norm(xh0, xl0);
        ff2_norm(xh1, xl1);
      }
    }
    ff2_norm(xh0, xl0);
    ff2_norm(xh1, xl1);
    emit(o, ff{xh0.x, xl0.x});
    emit(o + 1, ff{xh0.y, xl0.y});
    emit(o + 2, ff{xh1.x, xl1.x});
    emit(o + 3, ff{xh1.y, xl1.y});
  }
  for (size_t i = 4 * ng + tid; i < N; i += nthr) {  // ragged end
    ff x{0.f, 0.f};
    for (int k = 0; k < m; ++k) x = ff_fma(ff{cf[k].x, cf[k].y}, ff{Uh[(size_t)k * ld + i], Ul[(size_t)k * ld + i]}, x);
    emit(i, x);
  }
}

// SMs of the current device, cached per device ordinal (thread-safe: a
// benign race only stores the same value twice).
int device_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 1;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
      cudaGetLastError();
      v = 1;
    }
    cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

// Blocks of the streaming reduction kernels: four per SM, at most RB_MAX.
int red_blocks() { return std::min(RB_MAX, 4 * device_sms()); }

int grid_for(size_t n) {
  size_t b = (n + NT - 1) / NT;
  const size_t cap = (size_t)red_blocks();
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

size_t reduction_scratch_entries() { return (size_t)RB_MAX * (2 * MMAX + 4) + 64; }

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

cudaError_t launch_norms(bool use_ff, KState* ks, void* part, int nx, const Vec* x, size_t n, int dev_P,
                         cudaStream_t s) {
  if (nx > NORMS_MAX || dev_P >= nx) return cudaErrorInvalidValue;
  LinArgs la{};
  la.nx = nx;
  la.n = n;
  la.dev_P = dev_P;
  for (int k = 0; k < nx; ++k) la.x[k] = x[k];
  const int g = grid_for(n);
  const size_t smem = (size_t)NORMS_MAX * g * 8;
  if (use_ff)
    k_norms<true><<<g, NT, smem, s>>>(ks, static_cast<ff*>(part), la);
  else
    k_norms<false><<<g, NT, smem, s>>>(ks, static_cast<double*>(part), la);
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
namespace {
__global__ void k_f64_to_fx(float2* out, const double* x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
    const ff f = ff_from_double(x[i]);
    out[i] = make_float2(f.h, f.l);
  }
}
}  // namespace

cudaError_t launch_f64_to_fx(float* out, const double* x, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_f64_to_fx<<<grid_for(n), NT, 0, s>>>(reinterpret_cast<float2*>(out), x, n);
  return cudaGetLastError();
}

cudaError_t launch_ff_to_f64(double* out, Vec x, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_ff_to_f64<<<grid_for(n), NT, 0, s>>>(out, x, n);
  return cudaGetLastError();
}

cudaError_t launch_start(bool use_ff, KState* ks, Basis U, Vec b0, size_t N, int P, double eta, double s0,
                         double alpha, int mode, cudaStream_t s) {
  const int g = grid_for(N + P);
  if (use_ff)
    k_start<true><<<g, NT, 0, s>>>(ks, U.at(0), b0, N, P, eta, s0, alpha, mode);
  else
    k_start<false><<<g, NT, 0, s>>>(ks, U.at(0), b0, N, P, eta, s0, alpha, mode);
  return cudaGetLastError();
}

cudaError_t launch_dots(bool use_ff, KState* ks, void* part, Basis U, int j, size_t n_aug, cudaStream_t s) {
  if (j < 0 || j + 1 > MMAX) return cudaErrorInvalidValue;
  const int ch = use_ff ? FF_CH : DOT_CHUNK;
  const int chunks = (j + 1 + ch - 1) / ch;
  int gx = (red_blocks() + chunks - 1) / chunks;
  const int need = (int)((n_aug / 4 + NT - 1) / NT);
  if (gx > need) gx = need;
  if (gx < 1) gx = 1;
  dim3 grid(gx, chunks);
  const size_t smem = (size_t)(2 * (j + 1) + 1) * gx * 8;
  const dim3 grid1((unsigned)(gx * chunks));  // float-float kernel: chunk-fastest 1D grid
  // thread-safe one-time set-up (function-local static initialisation)
  static const cudaError_t configured = [] {
    // (2 MMAX + 1) partials of up to RB_MAX / chunks blocks each, 8 bytes
    cudaError_t e = cudaFuncSetAttribute(k_dots_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_dots<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    return e;
  }();
  if (configured != cudaSuccess) return configured;
  if (use_ff) return pdl_launch(k_dots_ff, grid1, dim3(NT), smem, s, ks, static_cast<ff*>(part), U, j, n_aug);
  return pdl_launch(k_dots<false>, grid, dim3(NT), smem, s, ks, static_cast<double*>(part), U, j, n_aug);
}

cudaError_t launch_update(bool use_ff, KState* ks, void* part, Basis U, int j, size_t n_aug, cudaStream_t s) {
  if (j < 0 || j + 1 > MMAX) return cudaErrorInvalidValue;
  if (use_ff) {
    const size_t tiles = (n_aug / 4 + UQB - 1) / UQB;
    const size_t cap = (size_t)std::min(RB_MAX, 3 * device_sms());
    const int g = (int)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
    return pdl_launch(k_update_ff, dim3(g), dim3(NT), (size_t)g * 8, s, ks, static_cast<ff*>(part), U, j, n_aug);
  }
  const int g = grid_for(n_aug / 4 + 1);
  return pdl_launch(k_update<false>, dim3(g), dim3(NT), (size_t)g * 8, s, ks, static_cast<double*>(part), U, j, n_aug);
}

namespace {

// One full wave of kernel Kern (its resident blocks on every SM with
// smem_max bytes of dynamic shared memory each), capped at red_blocks() (the
// partial-sum scratch and the update's staging hold that many per row) and at
// `need`.  Measured once per kernel (thread-safe static initialisation;
// smem_max is a constant of the kernel, and the kernel's dynamic shared memory
// limit must already admit it).
template <auto Kern>
int one_wave(size_t need, size_t smem_max) {
  static const int wave = [smem_max] {
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, Kern, NT, smem_max);
    return std::min(red_blocks(), std::max(1, nsm) * std::max(1, occ));
  }();
  return (int)std::max<size_t>(std::min(need, (size_t)wave), 1);
}

// Blocks of the incomplete-orthogonalisation passes: at least IOM_QUADS
// quads (4 entries) per thread.  Every block of the update sums all the
// products pass's per-block partials (FP64 additions on GB300's narrow FP64
// pipe), so on a small problem fewer, fuller blocks halve that work; a large
// problem fills the wave (red_blocks()) either way.
constexpr size_t IOM_QUADS = 4;
inline size_t iom_need(size_t n_aug) { return (n_aug / 4 + NT * IOM_QUADS - 1) / (NT * IOM_QUADS); }

template <int KW>
int iom_dots_grid(int kf, size_t n_aug) {
  const size_t need = iom_need(n_aug);
  if (kf == KF_FF) return one_wave<k_iom_dots_ff<KW>>(need, 0);
  if (kf == KF_MX) return one_wave<k_iom_dots_mx<KW>>(need, 0);
  return one_wave<k_iom_dots<KW>>(need, 0);
}
// the update's dynamic shared memory stages (KW + 1) Gd + Gu partials, Gd, Gu <= red_blocks()
template <int KW>
size_t iom_update_smem_max() {
  return (size_t)(KW + 2) * red_blocks() * 8;
}
// Raise the update kernels' dynamic shared memory limit to that (once; before
// any occupancy query or launch).
template <int KW>
cudaError_t iom_update_configure() {
  static const cudaError_t configured = [] {
    const int mx = (int)iom_update_smem_max<KW>();
    cudaError_t e = cudaFuncSetAttribute(k_iom_update_ff<KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_iom_update<KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_iom_update_mx<KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return e;
  }();
  return configured;
}
template <int KW>
int iom_update_grid(int kf, size_t n_aug) {
  const size_t need = iom_need(n_aug);
  if (iom_update_configure<KW>() != cudaSuccess) return 1;
  const size_t smem = iom_update_smem_max<KW>();
  if (kf == KF_FF) return one_wave<k_iom_update_ff<KW>>(need, smem);
  if (kf == KF_MX) return one_wave<k_iom_update_mx<KW>>(need, smem);
  return one_wave<k_iom_update<KW>>(need, smem);
}

template <int KW>
cudaError_t iom_dots_kw(int kf, KState* ks, void* part, Basis U, int j, size_t N, size_t n_aug, cudaStream_t s) {
  const int g = iom_dots_grid<KW>(kf, n_aug);
  if (kf == KF_FF)
    return pdl_launch(k_iom_dots_ff<KW>, dim3(g), dim3(NT), 0, s, ks, static_cast<ff*>(part), U, j, n_aug);
  if (kf == KF_MX)
    return pdl_launch(k_iom_dots_mx<KW>, dim3(g), dim3(NT), 0, s, ks, static_cast<double*>(part), U, j, N, n_aug);
  return pdl_launch(k_iom_dots<KW>, dim3(g), dim3(NT), 0, s, ks, static_cast<double*>(part), U, j, n_aug);
}

template <int KW>
cudaError_t iom_update_kw(int kf, KState* ks, void* part, Basis U, int j, size_t N, size_t n_aug, cudaStream_t s) {
  const cudaError_t configured = iom_update_configure<KW>();
  if (configured != cudaSuccess) return configured;
  const int gd = iom_dots_grid<KW>(kf, n_aug), g = iom_update_grid<KW>(kf, n_aug);
  const size_t smem = (size_t)((KW + 1) * gd + g) * 8;
  if (kf == KF_FF)
    return pdl_launch(k_iom_update_ff<KW>, dim3(g), dim3(NT), smem, s, ks, static_cast<ff*>(part), U, j, n_aug, gd);
  if (kf == KF_MX)
    return pdl_launch(k_iom_update_mx<KW>, dim3(g), dim3(NT), smem, s, ks, static_cast<double*>(part), U, j, N,
                      n_aug, gd);
  return pdl_launch(k_iom_update<KW>, dim3(g), dim3(NT), smem, s, ks, static_cast<double*>(part), U, j, n_aug, gd);
}

}  // namespace

cudaError_t launch_iom_dots(int kf, int iop, KState* ks, void* part, Basis U, int j, size_t N, size_t n_aug,
                            cudaStream_t s) {
  if (j < 0 || j + 1 > MMAX) return cudaErrorInvalidValue;
  switch (iop) {
    case 1: return iom_dots_kw<1>(kf, ks, part, U, j, N, n_aug, s);
    case 2: return iom_dots_kw<2>(kf, ks, part, U, j, N, n_aug, s);
    case 3: return iom_dots_kw<3>(kf, ks, part, U, j, N, n_aug, s);
    case 4: return iom_dots_kw<4>(kf, ks, part, U, j, N, n_aug, s);
    case 5: return iom_dots_kw<5>(kf, ks, part, U, j, N, n_aug, s);
    case 6: return iom_dots_kw<6>(kf, ks, part, U, j, N, n_aug, s);
    case 7: return iom_dots_kw<7>(kf, ks, part, U, j, N, n_aug, s);
    case 8: return iom_dots_kw<8>(kf, ks, part, U, j, N, n_aug, s);
    default: return cudaErrorInvalidValue;
  }
}

int iom_update_blocks(int kf, int iop, size_t n_aug) {
  switch (iop) {
    case 1: return iom_update_grid<1>(kf, n_aug);
    case 2: return iom_update_grid<2>(kf, n_aug);
    case 3: return iom_update_grid<3>(kf, n_aug);
    case 4: return iom_update_grid<4>(kf, n_aug);
    case 5: return iom_update_grid<5>(kf, n_aug);
    case 6: return iom_update_grid<6>(kf, n_aug);
    case 7: return iom_update_grid<7>(kf, n_aug);
    case 8: return iom_update_grid<8>(kf, n_aug);
    default: return 0;
  }
}

cudaError_t launch_iom_update(int kf, int iop, KState* ks, void* part, Basis U, int j, size_t N, size_t n_aug,
                              cudaStream_t s) {
  if (j < 0 || j + 1 > MMAX) return cudaErrorInvalidValue;
  switch (iop) {
    case 1: return iom_update_kw<1>(kf, ks, part, U, j, N, n_aug, s);
    case 2: return iom_update_kw<2>(kf, ks, part, U, j, N, n_aug, s);
    case 3: return iom_update_kw<3>(kf, ks, part, U, j, N, n_aug, s);
    case 4: return iom_update_kw<4>(kf, ks, part, U, j, N, n_aug, s);
    case 5: return iom_update_kw<5>(kf, ks, part, U, j, N, n_aug, s);
    case 6: return iom_update_kw<6>(kf, ks, part, U, j, N, n_aug, s);
    case 7: return iom_update_kw<7>(kf, ks, part, U, j, N, n_aug, s);
    case 8: return iom_update_kw<8>(kf, ks, part, U, j, N, n_aug, s);
    default: return cudaErrorInvalidValue;
  }
}

// One phi kernel instantiation, launched as clusters of `cl` CTAs.
template <typename T, int GROUPS>
cudaError_t phi_launch(int cl, size_t smem, cudaStream_t s, KState* ks, int m, double beta, double tol, int force,
                       int diff_rule, const void* iom_part, int iom_kf, int iom_gu, int pair, const PhiConst& pc) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(cl);
  lc.blockDim = dim3(PHI_NT);
  lc.dynamicSmemBytes = smem;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, k_phi<T, GROUPS>, ks, m, beta, tol, force, diff_rule, iom_part, iom_kf, iom_gu, pair,
                            pc);
}

template <typename T>
cudaError_t phi_configure(int smax) {
  cudaError_t e = cudaFuncSetAttribute(k_phi<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_phi<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_phi<T, 2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

// Whether clusters of 2 PHI_CL CTAs with the largest shared memory fit the GPU.
template <typename T>
bool phi_two_groups_fit(int smax) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(2 * PHI_CL);
  lc.blockDim = dim3(PHI_NT);
  lc.dynamicSmemBytes = smax;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2 * PHI_CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_phi<T, 2>, &lc) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

cudaError_t launch_phi(KState* ks, int m, double beta, double tol, int force_accept, int diff_rule,
                       const void* iom_part, int iom_kf, int iom_gu, bool ff_arith, bool pair, cudaStream_t s) {
  if (m < 1 || m > MMAX) return cudaErrorInvalidValue;
  static const PhiConst pc = [] {
    PhiConst c{};
    double f = 1.0;
    for (int k = 0; k <= 18; ++k) {
      if (k > 0) f /= k;
      const float h = (float)f;
      c.d[k] = f;
      c.f[k] = make_float2(h, (float)(f - (double)h));
    }
    return c;
  }();
  static_assert(sizeof(double) == sizeof(ff), "the two forms use the same shared memory");
  const int smax = (int)(6 * sizeof(double) *
                         std::max(MMAX * MMAX, PHI_PAIR_MAX * PHI_PAIR_MAX + (PHI_PAIR_MAX - 1) * (PHI_PAIR_MAX - 1)));
  static const cudaError_t configured = [smax] {
    cudaError_t e = phi_configure<double>(smax);
    if (e == cudaSuccess) e = phi_configure<ff>(smax);
    return e;
  }();
  if (configured != cudaSuccess) return configured;
  // the pair on two groups of CTAs (one matrix each) where such clusters fit,
  // else packed on one group up to m = PHI_PAIR_MAX
  static const bool two_fit = phi_two_groups_fit<ff>(6 * (int)sizeof(double) * MMAX * MMAX) &&
                              phi_two_groups_fit<double>(6 * (int)sizeof(double) * MMAX * MMAX);
  pair = pair && m >= 2;
  const bool two_groups = pair && two_fit;
  pair = pair && (two_groups || m <= PHI_PAIR_MAX);
  const size_t smem =
      6 * sizeof(double) * ((size_t)m * m + (pair && !two_groups ? (size_t)(m - 1) * (m - 1) : 0));
  const int cl = two_groups ? 2 * PHI_CL : PHI_CL;
  if (ff_arith)
    return two_groups ? phi_launch<ff, 2>(cl, smem, s, ks, m, beta, tol, force_accept, diff_rule, iom_part, iom_kf,
                                          iom_gu, 1, pc)
                      : phi_launch<ff, 1>(cl, smem, s, ks, m, beta, tol, force_accept, diff_rule, iom_part, iom_kf,
                                          iom_gu, pair ? 1 : 0, pc);
  return two_groups ? phi_launch<double, 2>(cl, smem, s, ks, m, beta, tol, force_accept, diff_rule, iom_part, iom_kf,
                                            iom_gu, 1, pc)
                    : phi_launch<double, 1>(cl, smem, s, ks, m, beta, tol, force_accept, diff_rule, iom_part, iom_kf,
                                            iom_gu, pair ? 1 : 0, pc);
}

cudaError_t launch_combine(bool use_ff, const KState* ks, Basis U, Vec base, Vec out, size_t N, bool if_accepted,
                           cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  if (use_ff)
    k_combine_ff<<<grid_for(N / 4 + 1), NT, 0, s>>>(ks, U, base, out, N, if_accepted ? 1 : 0);
  else
    k_combine<false><<<grid_for(N), NT, 0, s>>>(ks, U, base, out, N, if_accepted ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace expdg
