// Nodal DG operator kernels: R(q) and the frozen-flux linear operator L(qt) v.
//
// Discretisation (paper Sec. 2.2 Eq. EXPO-SemiDiscretizedForm_ode, Sec. 3.1,
// Sec. 3.2; LGL collocation, Sec. 4): on each tensor-product element,
//
//   R = - sum_d (2/h_d) D^(d) F_d  -  (2/h_d)(1/w_0) (F*.n - F^-.n) at face nodes,
//   F*.n = 1/2 (F^- + F^+).n + 1/2 lambda (q^- - q^+)       (Lax-Friedrichs),
//
// with lambda = max(|u^-|, |u^+|) for Burgers (Sec. 3.1) and
// max(|u^-.n| + a^-, |u^+.n| + a^+) for Euler (Sec. 5.1).  The linear operator
// replaces F_d(q) by A_d(qt) v (Eq. linearflux) and q^-/q^+ in the jump by
// v^-/v^+, with lambda taken from qt (frozen).
//
// Kernel layout: one CTA holds EPB consecutive elements, one thread per node.
// A thread loads its own node (coalesced: the canonical layout keeps the
// nodes of consecutive elements contiguous per field), writes its d-fluxes
// to shared memory, then forms the tensor-product derivative from the fluxes
// of its line and, on face nodes, the numerical flux with the neighbour's
// trace read from global memory (L2-resident: the neighbour element is
// being processed by the same or a nearby CTA).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "ff.cuh"

namespace expdg {

template <int DIM, int EQ>
struct NFields {
  static constexpr int value = (EQ == EXPDG_BURGERS) ? 1 : DIM + 2;
};

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Elements per CTA: about 256 threads.
template <int DIM, int P>
__host__ __device__ constexpr int elems_per_block() {
  return (256 / ipow(P + 1, DIM)) > 0 ? (256 / ipow(P + 1, DIM)) : 1;
}

// ---------------------------------------------------------------- physics ---
template <int DIM, int EQ, typename T>
struct Phys {
  static constexpr int M = NFields<DIM, EQ>::value;

  __device__ __forceinline__ static T pressure(const T* q, T gm1) {
    T inv = T(1) / q[0];
    T ke = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) ke += q[1 + k] * q[1 + k];
    return gm1 * (q[DIM + 1] - T(0.5) * ke * inv);
  }

  // physical flux F_d(q)
  __device__ __forceinline__ static void flux(const T* q, int d, T gm1, T* F) {
    if (EQ == EXPDG_BURGERS) {
      F[0] = T(0.5) * q[0] * q[0];
      return;
    }
    T inv = T(1) / q[0];
    T ud = q[1 + d] * inv;
    T p = pressure(q, gm1);
    F[0] = q[1 + d];
#pragma unroll
    for (int k = 0; k < DIM; ++k) F[1 + k] = q[1 + k] * ud + (k == d ? p : T(0));
    F[DIM + 1] = (q[DIM + 1] + p) * ud;
  }

  // A_d(qt) v: directional derivative of F_d at qt along v
  __device__ __forceinline__ static void jac(const T* qt, const T* v, int d, T gm1, T* F) {
    if (EQ == EXPDG_BURGERS) {
      F[0] = qt[0] * v[0];
      return;
    }
    T inv = T(1) / qt[0];
    T u[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) u[k] = qt[1 + k] * inv;
    T uu = T(0), udm = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      uu += u[k] * u[k];
      udm += u[k] * v[1 + k];
    }
    T p = gm1 * (qt[DIM + 1] - T(0.5) * qt[0] * uu);
    T dp = gm1 * (v[DIM + 1] - udm + T(0.5) * uu * v[0]);
    T dud = (v[1 + d] - u[d] * v[0]) * inv;  // delta u_d
    F[0] = v[1 + d];
#pragma unroll
    for (int k = 0; k < DIM; ++k) F[1 + k] = v[1 + k] * u[d] + qt[1 + k] * dud + (k == d ? dp : T(0));
    F[DIM + 1] = (v[DIM + 1] + dp) * u[d] + (qt[DIM + 1] + p) * dud;
  }

  // |u.e_d| + a  (Euler), |u| (Burgers)
  __device__ __forceinline__ static T wave(const T* q, int d, T gamma) {
    if (EQ == EXPDG_BURGERS) return fabs(q[0]);
    T inv = T(1) / q[0];
    T p = pressure(q, gamma - T(1));
    return fabs(q[1 + d] * inv) + sqrt(gamma * p * inv);
  }

  __device__ __forceinline__ static bool physical(const T* q, T gamma) {
    if (EQ == EXPDG_BURGERS) return true;
    return q[0] > T(0) && pressure(q, gamma - T(1)) > T(0);
  }
};

// LINEAR = false: residual; true: linear operator.  T = double: FP64 form
// (double in, double out); T = float: mixed form (float in, float-float out).
template <int DIM, int P, int EQ, typename T, bool LINEAR>
__global__ void __launch_bounds__(ipow(P + 1, DIM) * elems_per_block<DIM, P>() <= 256 ? 256 : 1024)
k_dg(const DGArgs a, const Tab tab) {
  constexpr int NP1 = P + 1;
  constexpr int NP = ipow(NP1, DIM);
  constexpr int M = NFields<DIM, EQ>::value;
  constexpr int EPB = elems_per_block<DIM, P>();
  constexpr int SLOT = EPB * NP;  // nodes held by the CTA
  constexpr bool FF = !std::is_same<T, double>::value;
  using PH = Phys<DIM, EQ, T>;

  griddep_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sF = reinterpret_cast<T*>(smem_raw);  // [DIM][M][SLOT]
  T* sD = sF + DIM * M * SLOT;             // [NP1][NP1]

  const int tid = threadIdx.x;
  for (int k = tid; k < NP1 * NP1; k += blockDim.x) sD[k] = (T)tab.D[k];

  const int e0 = blockIdx.x * EPB;
  const int le = tid / NP;
  const int n = tid - le * NP;
  const int e = e0 + le;
  const bool active = (tid < SLOT) && (e < a.nelem);
  const T gamma = (T)a.gamma;
  const T gm1 = gamma - T(1);
  const size_t stride = a.stride;
  const T* __restrict__ qin = static_cast<const T*>(a.q);
  const T* __restrict__ vin = static_cast<const T*>(a.v);

  T qv[M];  // residual: q at the node; linear: qt at the node
  T vv[M];  // linear: v at the node
  if (active) {
    const size_t base = (size_t)e * NP + n;
#pragma unroll
    for (int f = 0; f < M; ++f) {
      qv[f] = qin[f * stride + base];
      if (LINEAR) vv[f] = vin[f * stride + base];
    }
    if (!LINEAR && !PH::physical(qv, gamma)) atomicOr(a.status, 1);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      T F[M];
      if (LINEAR)
        PH::jac(qv, vv, d, gm1, F);
      else
        PH::flux(qv, d, gm1, F);
#pragma unroll
      for (int f = 0; f < M; ++f) sF[(d * M + f) * SLOT + tid] = F[f];
    }
  }
  __syncthreads();
  griddep_launch();
  if (!active) return;

  int ii[DIM];
  {
    int t = n;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      ii[d] = t % NP1;
      t /= NP1;
    }
  }
  int ec[3] = {0, 0, 0};
  {
    int t = e;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      ec[d] = t % a.ne[d];
      t /= a.ne[d];
    }
  }

  T acc[M];
#pragma unroll
  for (int f = 0; f < M; ++f) acc[f] = T(0);
  const T lift = (T)tab.lift;

#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int sd = (d == 0) ? 1 : (d == 1 ? NP1 : NP1 * NP1);
    const T c2h = (T)a.two_over_h[d];
    const int lbase = tid - ii[d] * sd;
    const T* Drow = sD + ii[d] * NP1;
#pragma unroll
    for (int f = 0; f < M; ++f) {
      const T* Fl = sF + (d * M + f) * SLOT + lbase;
      T sum = T(0);
#pragma unroll
      for (int j = 0; j < NP1; ++j) sum += Drow[j] * Fl[j * sd];
      acc[f] -= c2h * sum;
    }
    if (ii[d] == 0 || ii[d] == P) {
      const int side = (ii[d] == 0) ? -1 : 1;
      int nc[3] = {ec[0], ec[1], ec[2]};
      nc[d] = nc[d] + side;
      if (nc[d] < 0) nc[d] += a.ne[d];
      if (nc[d] >= a.ne[d]) nc[d] -= a.ne[d];
      int en = nc[0];
      if (DIM > 1) en += a.ne[0] * (nc[1] + (DIM > 2 ? a.ne[1] * nc[2] : 0));
      const int nn = n + (side < 0 ? P : -P) * sd;
      const size_t nb = (size_t)en * NP + nn;
      T qn[M], vn[M], Fp[M], Fm[M];
#pragma unroll
      for (int f = 0; f < M; ++f) {
        qn[f] = qin[f * stride + nb];
        if (LINEAR) vn[f] = vin[f * stride + nb];
        Fm[f] = sF[(d * M + f) * SLOT + tid];
      }
      if (LINEAR)
        PH::jac(qn, vn, d, gm1, Fp);
      else
        PH::flux(qn, d, gm1, Fp);
      const T lam = fmax(PH::wave(qv, d, gamma), PH::wave(qn, d, gamma));
      const T sgn = (T)side;
#pragma unroll
      for (int f = 0; f < M; ++f) {
        const T jump = LINEAR ? (vv[f] - vn[f]) : (qv[f] - qn[f]);
        const T fstar_n = T(0.5) * (Fm[f] + Fp[f]) * sgn + T(0.5) * lam * jump;
        acc[f] -= c2h * lift * (fstar_n - Fm[f] * sgn);
      }
    }
  }

  const size_t base = (size_t)e * NP + n;
  const bool aug = LINEAR && a.paug > 0 && (FF ? a.tail_h != nullptr : a.tail_d != nullptr);
  if constexpr (!FF) {
    const double vs = (LINEAR && a.vs_d != nullptr) ? *a.vs_d : 1.0;
    const double scale = a.alpha * vs;
    double cf[EXPDG_MAX_PHI];
    bool any = false;
#pragma unroll
    for (int k = 0; k < EXPDG_MAX_PHI; ++k) {
      cf[k] = (aug && k < a.paug) ? a.eta * vs * a.tail_d[k] : 0.0;
      any |= (cf[k] != 0.0);
    }
#pragma unroll
    for (int f = 0; f < M; ++f) {
      double o = scale * (double)acc[f];
      if (any) {
        const size_t gi = f * stride + base;
#pragma unroll
        for (int k = 1; k <= EXPDG_MAX_PHI; ++k)
          if (k <= a.paug && cf[k - 1] != 0.0) o += cf[k - 1] * a.W_d[a.paug + 1 - k][gi];
      }
      a.out[f * stride + base] = o;
    }
    if (aug && blockIdx.x == 0 && tid == 0)
      for (int k = 0; k < a.paug; ++k) a.out_tail_d[k] = (k + 1 < a.paug) ? vs * a.tail_d[k + 1] : 0.0;
  } else {
    const ff vs = (LINEAR && a.vs_h != nullptr) ? ff{*a.vs_h, *a.vs_l} : ff{1.0f, 0.0f};
    const ff scale = ff_mul(ff{a.alpha_h, a.alpha_l}, vs);
    ff cf[EXPDG_MAX_PHI];
    bool any = false;
#pragma unroll
    for (int k = 0; k < EXPDG_MAX_PHI; ++k) {
      cf[k] = ff{0.0f, 0.0f};
      if (aug && k < a.paug) {
        ff t = ff_mul(vs, ff{a.tail_h[k], a.tail_l[k]});
        const float eta = (float)a.eta;  // a power of two: exact
        cf[k] = ff{t.h * eta, t.l * eta};
      }
      any |= (cf[k].h != 0.0f);
    }
#pragma unroll
    for (int f = 0; f < M; ++f) {
      // exact float * float-float product, then the augmentation in float-float
      float p = __fmul_rn((float)acc[f], scale.h);
      float pe = __fmaf_rn((float)acc[f], scale.h, -p);
      pe = __fmaf_rn((float)acc[f], scale.l, pe);
      ff o = ff_fast_two_sum(p, pe);
      if (any) {
        const size_t gi = f * stride + base;
#pragma unroll
        for (int k = 1; k <= EXPDG_MAX_PHI; ++k)
          if (k <= a.paug && cf[k - 1].h != 0.0f) {
            const int wi = a.paug + 1 - k;
            o = ff_fma(cf[k - 1], ff{a.W_h[wi][gi], a.W_l[wi][gi]}, o);
          }
      }
      a.out_h[f * stride + base] = o.h;
      a.out_l[f * stride + base] = o.l;
    }
    if (aug && blockIdx.x == 0 && tid == 0)
      for (int k = 0; k < a.paug; ++k) {
        ff t = (k + 1 < a.paug) ? ff_mul(vs, ff{a.tail_h[k + 1], a.tail_l[k + 1]}) : ff{0.0f, 0.0f};
        a.out_tail_h[k] = t.h;
        a.out_tail_l[k] = t.l;
      }
  }
}

template <int DIM, int P, int EQ, typename T, bool LINEAR>
cudaError_t launch_dg_t(const DGArgs& a, const Tab& t, cudaStream_t s) {
  constexpr int NP = ipow(P + 1, DIM);
  constexpr int M = NFields<DIM, EQ>::value;
  constexpr int EPB = elems_per_block<DIM, P>();
  const int threads = ((EPB * NP + 31) / 32) * 32;
  const size_t smem = sizeof(T) * ((size_t)DIM * M * EPB * NP + (P + 1) * (P + 1));
  const int blocks = (a.nelem + EPB - 1) / EPB;
  auto kern = k_dg<DIM, P, EQ, T, LINEAR>;
  // once per instantiation, thread-safe (function-local static initialisation)
  static const cudaError_t configured =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (configured != cudaSuccess) return configured;
  if (blocks == 0) return cudaSuccess;
  return pdl_launch(kern, dim3(blocks), dim3(threads), smem, s, a, t);
}

template <int DIM, int EQ, typename T, bool LINEAR>
cudaError_t launch_dg_p(int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  switch (p) {
    case 1: return launch_dg_t<DIM, 1, EQ, T, LINEAR>(a, t, s);
    case 2: return launch_dg_t<DIM, 2, EQ, T, LINEAR>(a, t, s);
    case 3: return launch_dg_t<DIM, 3, EQ, T, LINEAR>(a, t, s);
    case 4: return launch_dg_t<DIM, 4, EQ, T, LINEAR>(a, t, s);
    case 5: return launch_dg_t<DIM, 5, EQ, T, LINEAR>(a, t, s);
    case 6: return launch_dg_t<DIM, 6, EQ, T, LINEAR>(a, t, s);
    case 7: return launch_dg_t<DIM, 7, EQ, T, LINEAR>(a, t, s);
    case 8: return launch_dg_t<DIM, 8, EQ, T, LINEAR>(a, t, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int DIM, int EQ>
cudaError_t launch_dg_dim(bool linear, bool fp32, int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  if (fp32)
    return linear ? launch_dg_p<DIM, EQ, float, true>(p, a, t, s) : launch_dg_p<DIM, EQ, float, false>(p, a, t, s);
  return linear ? launch_dg_p<DIM, EQ, double, true>(p, a, t, s) : launch_dg_p<DIM, EQ, double, false>(p, a, t, s);
}

}  // namespace expdg
