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
#include "cvt.cuh"
#include "ff.cuh"
#include "fx.cuh"

namespace expdg {

// A constant (or an entry of D) in the compute type T.
template <typename T>
__device__ __forceinline__ T cst(const Cst& c);
template <>
__device__ __forceinline__ double cst<double>(const Cst& c) { return c.d; }
template <>
__device__ __forceinline__ float cst<float>(const Cst& c) { return c.h; }
template <>
__device__ __forceinline__ fx cst<fx>(const Cst& c) { return fx(c.h, c.l); }
template <typename T>
__device__ __forceinline__ T d_entry(const Tab& t, int k) {
  if constexpr (std::is_same<T, double>::value) return t.D[k];
  else if constexpr (std::is_same<T, float>::value) return t.Dh[k];
  else return fx(t.Dh[k], t.Dl[k]);
}

template <int DIM, int EQ>
struct NFields {
  static constexpr int value = (EQ == EXPDG_BURGERS) ? 1 : DIM + 2;
};

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Elements per CTA for tile class TK (tile_threads): at least one element.
template <int DIM, int P, int TK = 0>
__host__ __device__ constexpr int elems_per_block() {
  return (tile_threads(TK) / ipow(P + 1, DIM)) > 0 ? (tile_threads(TK) / ipow(P + 1, DIM)) : 1;
}
// Threads per CTA: one per node of its elements, whole warps.
template <int DIM, int P, int TK = 0>
__host__ __device__ constexpr int dg_threads() {
  return ((elems_per_block<DIM, P, TK>() * ipow(P + 1, DIM) + 31) / 32) * 32;
}

// ---------------------------------------------------------------- physics ---
// Residual: fluxes from the primitive variables, computed once per state.
// Linear operator: A_d(qt) v from the linearisation state z of qt, computed
// once per step by k_linstate (Euler: z = (u_1..u_DIM, H, a) with the total
// enthalpy H = (E + p) / rho and the sound speed a; Burgers: z = qt), so the
// operator applies take no division and no square root.  With u_d and
// du_d = (v_{m_d} - u_d v_rho) / rho,
//   A_d v = ( v_{m_d},  v_{m_k} u_d + rho u_k du_d + delta_kd dp,
//             (v_E + dp) u_d + (E + p) du_d ),
//   dp = (gamma - 1) (v_E - u.v_m + |u|^2 v_rho / 2),
// and rho u_k du_d = u_k (v_{m_d} - u_d v_rho), (E + p) du_d = H (v_{m_d} - u_d v_rho).
template <int DIM, int EQ, typename T>
struct Phys {
  static constexpr int M = NFields<DIM, EQ>::value;
  static constexpr bool EULER = EQ == EXPDG_EULER;

  struct Prim {
    T u[DIM];  // velocity (Burgers: the state)
    T p;       // pressure
    T a;       // sound speed
  };

  __device__ __forceinline__ static Prim prim(const T* q, T gamma) {
    Prim w;
    if (!EULER) {
      w.u[0] = q[0];
      w.p = T(0);
      w.a = T(0);
      return w;
    }
    const T inv = T(1) / q[0];
    T ke = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      w.u[k] = q[1 + k] * inv;
      ke += q[1 + k] * w.u[k];
    }
    w.p = (gamma - T(1)) * (q[DIM + 1] - T(0.5) * ke);
    w.a = sqrt(gamma * w.p * inv);
    return w;
  }

  __device__ __forceinline__ static bool physical(const T* q, const Prim& w) {
    return !EULER || (q[0] > T(0) && w.p > T(0));
  }

  // physical flux F_d(q)
  __device__ __forceinline__ static void flux(const T* q, const Prim& w, int d, T* F) {
    if (!EULER) {
      F[0] = T(0.5) * q[0] * q[0];
      return;
    }
    const T ud = w.u[d];
    F[0] = q[1 + d];
#pragma unroll
    for (int k = 0; k < DIM; ++k) F[1 + k] = q[1 + k] * ud + (k == d ? w.p : T(0));
    F[DIM + 1] = (q[DIM + 1] + w.p) * ud;
  }

  // |u.e_d| + a  (Euler), |u| (Burgers)
  __device__ __forceinline__ static T wave(const Prim& w, int d) {
    return EULER ? fabs(w.u[d]) + w.a : fabs(w.u[0]);
  }

  // pressure perturbation dp of v at the linearisation state z (0 for Burgers)
  __device__ __forceinline__ static T lin_dp(const T* z, const T* v, T gm1) {
    if (!EULER) return T(0);
    T uu = T(0), uv = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      uu += z[k] * z[k];
      uv += z[k] * v[1 + k];
    }
    return gm1 * (v[DIM + 1] - uv + T(0.5) * uu * v[0]);
  }

  // A_d(qt) v
  __device__ __forceinline__ static void lin_flux(const T* z, const T* v, T dp, int d, T* F) {
    if (!EULER) {
      F[0] = z[0] * v[0];
      return;
    }
    const T ud = z[d];
    const T du = v[1 + d] - ud * v[0];  // rho du_d
    F[0] = v[1 + d];
#pragma unroll
    for (int k = 0; k < DIM; ++k) F[1 + k] = v[1 + k] * ud + z[k] * du + (k == d ? dp : T(0));
    F[DIM + 1] = (v[DIM + 1] + dp) * ud + z[DIM] * du;
  }

  __device__ __forceinline__ static T lin_wave(const T* z, int d) {
    return EULER ? fabs(z[d]) + z[DIM + 1] : fabs(z[0]);
  }

  // Roe dissipation |A(q*_Roe)| dq in direction e_d (Sec. 3.2): the Roe
  // average of two states given by velocity, total enthalpy and sqrt(rho),
  // then the waves of the flux Jacobian at (u*, H*): acoustic u_n -+ a with
  // strengths (dp -+ a (dm_n - u_n drho)) / (2 a^2), entropy u_n with
  // drho - dp / a^2, shear u_n with dm_t - u_t drho, where
  // dp = (gamma - 1)(dE - u.dm + |u|^2 drho / 2); right eigenvectors
  // (1, u -+ a e_d, H -+ u_n a), (1, u, |u|^2 / 2), (0, e_t, u_t).
  __device__ __forceinline__ static void roe_dissipation(const T* uL, T HL, T sL, const T* uR, T HR, T sR, const T* dq,
                                                         int d, T gm1, T* out) {
    const T inv = T(1) / (sL + sR);
    T u[DIM];
    T uu = T(0), udm = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      u[k] = (sL * uL[k] + sR * uR[k]) * inv;
      uu += u[k] * u[k];
      udm += u[k] * dq[1 + k];
    }
    const T H = (sL * HL + sR * HR) * inv;
    const T a2 = gm1 * (H - T(0.5) * uu);
    const T a = sqrt(a2), ia2 = T(1) / a2;
    const T un = u[d];
    const T dr = dq[0];
    const T dp = gm1 * (dq[DIM + 1] - udm + T(0.5) * uu * dr);
    const T dun = dq[1 + d] - un * dr;
    const T wm = fabs(un - a) * T(0.5) * (dp - a * dun) * ia2;
    const T wp = fabs(un + a) * T(0.5) * (dp + a * dun) * ia2;
    const T l0 = fabs(un), w0 = l0 * (dr - dp * ia2);
    const T ws = wm + w0 + wp;
    out[0] = ws;
    T shearE = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      if (k == d) {
        out[1 + k] = ws * u[k] + (wp - wm) * a;
      } else {
        const T st = dq[1 + k] - u[k] * dr;
        out[1 + k] = ws * u[k] + l0 * st;
        shearE += u[k] * st;
      }
    }
    out[DIM + 1] = (wm + wp) * H + (wp - wm) * un * a + w0 * T(0.5) * uu + l0 * shearE;
  }
};

// Linearisation state z of q (FP64 in, T out) at node i; stride =
// unknowns per field.  Computed in FP64 and rounded once.  Euler: (u, H, a),
// or (u, H, sqrt(rho)) for the Roe flux (its average weights).  qfx (may be
// null): q as float-float pairs as well (the mixed form's residual operand).
template <int DIM, int EQ, typename T>
__device__ __forceinline__ void linstate_node(const double* __restrict__ q, T* __restrict__ z, size_t stride,
                                              double gamma, int roe, float2* __restrict__ qfx, size_t i) {
  constexpr int M = NFields<DIM, EQ>::value;
  {
    double qv[M];
#pragma unroll
    for (int f = 0; f < M; ++f) qv[f] = q[f * stride + i];
    if (qfx != nullptr)  // the float-float split, conversions on the integer pipes
#pragma unroll
      for (int f = 0; f < M; ++f) {
        const float h = f64_to_f32_rn(qv[f]);
        qfx[f * stride + i] = make_float2(h, f64_to_f32_rn(qv[f] - f32_to_f64_exact(h)));
      }
    if (EQ != EXPDG_EULER) {
      if constexpr (std::is_same<T, float>::value)
        z[i] = f64_to_f32_rn(qv[0]);
      else
        z[i] = (T)qv[0];
    } else if constexpr (std::is_same<T, float>::value) {
      // FP32 state (mixed and float-float forms), few FP64 operations (on
      // GB300 the FP64 pipe runs about 1.6 lane operations per SM per clock):
      // 1/rho from the FP32 reciprocal and one Newton step in FP64 (relative
      // error about 2^-46), the pressure (where E and the kinetic energy may
      // cancel) in FP64, the sound speed's square root in FP32, conversions on
      // the integer pipes.  Each z entry is within about one FP32 rounding of
      // the FP64 value.
      const double r0 = f32_to_f64_exact(__frcp_rn(f64_to_f32_rn(qv[0])));
      const double inv = r0 * fma(-qv[0], r0, 2.0);
      double ke = 0.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double u = qv[1 + k] * inv;
        z[k * stride + i] = f64_to_f32_rn(u);
        ke = fma(qv[1 + k], u, ke);
      }
      const double p = (gamma - 1.0) * fma(-0.5, ke, qv[DIM + 1]);
      z[DIM * stride + i] = f64_to_f32_rn((qv[DIM + 1] + p) * inv);
      z[(DIM + 1) * stride + i] =
          __fsqrt_rn(f64_to_f32_rn(roe ? qv[0] : gamma * p * inv));
    } else {
      const double inv = 1.0 / qv[0];
      double ke = 0.0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double u = qv[1 + k] * inv;
        z[k * stride + i] = (T)u;
        ke += qv[1 + k] * u;
      }
      const double p = (gamma - 1.0) * (qv[DIM + 1] - 0.5 * ke);
      z[DIM * stride + i] = (T)((qv[DIM + 1] + p) * inv);
      z[(DIM + 1) * stride + i] = (T)(roe ? sqrt(qv[0]) : sqrt(gamma * p * inv));
    }
  }
}

template <int DIM, int EQ, typename T>
__global__ void __launch_bounds__(256) k_linstate(const double* __restrict__ q, T* __restrict__ z, size_t stride,
                                                  double gamma, int roe, float2* __restrict__ qfx) {
  griddep_wait();
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < stride) linstate_node<DIM, EQ, T>(q, z, stride, gamma, roe, qfx, i);
  griddep_launch();
}

template <int DIM, int EQ>
cudaError_t launch_linstate_dim(bool fp32, const double* q, void* z, size_t stride, double gamma, int roe,
                               float* qfx, cudaStream_t s) {
  if (stride == 0) return cudaSuccess;
  const dim3 grid((unsigned)((stride + 255) / 256));
  float2* qf = reinterpret_cast<float2*>(qfx);
  if (fp32)
    return pdl_launch(k_linstate<DIM, EQ, float>, grid, dim3(256), 0, s, q, static_cast<float*>(z), stride, gamma, roe,
                      qf);
  return pdl_launch(k_linstate<DIM, EQ, double>, grid, dim3(256), 0, s, q, static_cast<double*>(z), stride, gamma, roe,
                    qf);
}

// Neighbour element across each face of the CTA's EPB elements e0, e0+1, ...
// into sNb[EPB][2 DIM], face (d, side) at 2 d + (side > 0): periodic box, or
// -1 outside a Dirichlet end.
template <int DIM, int P, int TK>
__device__ __forceinline__ void build_neighbours(const DGArgs& a, int e0, int* sNb) {
  constexpr int EPB = elems_per_block<DIM, P, TK>(), NF = 2 * DIM;
  for (int k = threadIdx.x; k < EPB * NF; k += blockDim.x) {
    const int el = k / NF, d = (k - el * NF) >> 1, hi = k & 1;
    int t = e0 + el, ec[3] = {0, 0, 0};
#pragma unroll
    for (int dd = 0; dd < DIM; ++dd) {
      ec[dd] = t % a.ne[dd];
      t /= a.ne[dd];
    }
    int c = ec[d] + (hi ? 1 : -1);
    const bool outside = c < 0 || c >= a.ne[d];
    if (c < 0) c += a.ne[d];
    if (c >= a.ne[d]) c -= a.ne[d];
    ec[d] = c;
    sNb[k] = (outside && a.dirichlet) ? -1 : ec[0] + (DIM > 1 ? a.ne[0] * (ec[1] + (DIM > 2 ? a.ne[1] * ec[2] : 0)) : 0);
  }
}

// Derivative and face terms at node n of the CTA's element le (thread tid):
//   acc = - sum_d (2/h_d) ( [D^(d) F_d]_n + (1/w_0) (F*.n - F^-.n) at face nodes ),
// from the fluxes of the CTA's nodes in sF.  qv: own state (residual) or
// linearisation state z (linear); vv: own linear input; w: own primitive
// variables (residual); nb_q(f, gi), nb_v(f, gi): the state (residual) or
// linearisation state (linear) and the linear input of field f at node gi
// (index within the field plane) of a neighbour element, in the compute type.
// Outside a Dirichlet end the neighbour's state and input are the boundary
// data 0.
template <int DIM, int P, int EQ, typename T, bool LINEAR, bool ROE, int TK, class NbQ, class NbV>
__device__ __forceinline__ void node_terms(const DGArgs& a, T lift, NbQ nb_q, const T* sF,
                                           const T* sD, const int* sNb, int tid, int le, int n,
                                           const T (&qv)[NFields<DIM, EQ>::value],
                                           const T (&vv)[NFields<DIM, EQ>::value],
                                           const typename Phys<DIM, EQ, T>::Prim& w, NbV nb_v,
                                           T (&acc)[NFields<DIM, EQ>::value]) {
  constexpr int NP1 = P + 1, NP = ipow(NP1, DIM), M = NFields<DIM, EQ>::value;
  constexpr int SLOT = elems_per_block<DIM, P, TK>() * NP, NF = 2 * DIM;
  using PH = Phys<DIM, EQ, T>;
  const T gamma = cst<T>(a.gamma), gm1 = gamma - T(1);
  int ii[DIM];
  {
    int t = n;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      ii[d] = t % NP1;
      t /= NP1;
    }
  }
#pragma unroll
  for (int f = 0; f < M; ++f) acc[f] = T(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int sd = (d == 0) ? 1 : (d == 1 ? NP1 : NP1 * NP1);
    const T c2h = cst<T>(a.two_over_h[d]);
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
      const bool hi = ii[d] == P;
      const int en = sNb[le * NF + 2 * d + (hi ? 1 : 0)];
      const int nn = n + (hi ? -P : P) * sd;
      // Dirichlet ends exist only for Burgers: the Euler kernels keep plain loads
      const bool outside = (EQ == EXPDG_BURGERS) && en < 0;
      const size_t nb = (size_t)(outside ? 0 : en) * NP + nn;
      T qn[M], vn[M], Fp[M], Fm[M];
#pragma unroll
      for (int f = 0; f < M; ++f) {
        qn[f] = outside ? T(0) : nb_q(f, nb);
        if (LINEAR) vn[f] = outside ? T(0) : nb_v(f, nb);
        Fm[f] = sF[(d * M + f) * SLOT + tid];
      }
      T Dj[M];  // dissipation term: lam (q^- - q^+) (LF) or |A(q*_Roe)| (q^- - q^+) (Roe)
      T dq[M];
#pragma unroll
      for (int f = 0; f < M; ++f) dq[f] = LINEAR ? (vv[f] - vn[f]) : (qv[f] - qn[f]);
      if (LINEAR) {
        PH::lin_flux(qn, vn, PH::lin_dp(qn, vn, gm1), d, Fp);
        if constexpr (ROE) {  // z = (u, H, sqrt(rho)) on both sides
          PH::roe_dissipation(qv, qv[M - 2], qv[M - 1], qn, qn[M - 2], qn[M - 1], dq, d, gm1, Dj);
        } else {
          const T lam = fmax(PH::lin_wave(qv, d), PH::lin_wave(qn, d));
#pragma unroll
          for (int f = 0; f < M; ++f) Dj[f] = lam * dq[f];
        }
      } else {
        const typename PH::Prim wn = PH::prim(qn, gamma);
        PH::flux(qn, wn, d, Fp);
        if constexpr (ROE) {  // the Roe average of the two states (H = (E + p) / rho)
          PH::roe_dissipation(w.u, (qv[M - 1] + w.p) / qv[0], sqrt(qv[0]), wn.u, (qn[M - 1] + wn.p) / qn[0],
                              sqrt(qn[0]), dq, d, gm1, Dj);
        } else {
          const T lam = fmax(PH::wave(w, d), PH::wave(wn, d));
#pragma unroll
          for (int f = 0; f < M; ++f) Dj[f] = lam * dq[f];
        }
      }
      const T sgn = hi ? T(1) : T(-1);
#pragma unroll
      for (int f = 0; f < M; ++f) {
        const T fstar_n = T(0.5) * (Fm[f] + Fp[f]) * sgn + T(0.5) * Dj[f];
        acc[f] -= c2h * lift * (fstar_n - Fm[f] * sgn);
      }
    }
  }
}

// Diffusion part of the 1D viscous Burgers operator (Sec. 3.1, Eq. gov-burgers1d,
// central fluxes) at the thread's node:
//   kappa [ (2/h) D q + (2/h)(1/w_0) n (q** - q^-) ],
//   q = (2/h) D u + (2/h)(1/w_0) n (u** - u^-),   u** = {u},  q** = {q},
// at a Dirichlet end u** = 0 and q** = q^-.  uin: the operand (the state for
// R, the input vector for L) in the compute type.  The CTA forms q on its
// elements and one halo element on each side (sU, sQ: (EPB + 2)(P + 1) + 2
// entries each); every thread of the CTA must call it.
template <int P, typename T, int TK, typename U>
__device__ T visc_term(const DGArgs& a, const U* __restrict__ uin, const T* sD, T lift, T* sU, T* sQ, int e0,
                       int tid, int le, int n, bool active) {
  constexpr int NP1 = P + 1;
  constexpr int EPB = elems_per_block<1, P, TK>();
  constexpr int NH = (EPB + 2) * NP1;  // halo slots: elements e0 - 1 .. e0 + EPB
  const int ne = a.ne[0];
  const T c2h = cst<T>(a.two_over_h[0]);
  auto elem_val = [&](int ge, int i) -> T {  // u at node i of element ge (periodic / zero outside)
    if (ge < 0 || ge >= ne) {
      if (a.dirichlet) return T(0);
      ge = ((ge % ne) + ne) % ne;
    }
    return (T)uin[(size_t)ge * NP1 + i];
  };
  for (int k = tid; k < NH; k += blockDim.x) sU[k] = elem_val(e0 - 1 + k / NP1, k % NP1);
  if (tid == 0) sU[NH] = elem_val(e0 - 2, P);             // right end of element e0 - 2
  if (tid == 1) sU[NH + 1] = elem_val(e0 + EPB + 1, 0);  // left end of element e0 + EPB + 1
  __syncthreads();
  for (int k = tid; k < NH; k += blockDim.x) {
    const int kk = k / NP1, i = k - kk * NP1, ge = e0 - 1 + kk;
    T q = T(0);
#pragma unroll
    for (int jn = 0; jn < NP1; ++jn) q += sD[i * NP1 + jn] * sU[kk * NP1 + jn];
    q *= c2h;
    if (i == 0) {
      const T u0 = sU[kk * NP1], uo = (kk == 0) ? sU[NH] : sU[(kk - 1) * NP1 + P];
      const T us = (a.dirichlet && ge == 0) ? T(0) : T(0.5) * (u0 + uo);
      q -= c2h * lift * (us - u0);
    }
    if (i == P) {
      const T uP = sU[kk * NP1 + P], uo = (kk == EPB + 1) ? sU[NH + 1] : sU[(kk + 1) * NP1];
      const T us = (a.dirichlet && ge == ne - 1) ? T(0) : T(0.5) * (uP + uo);
      q += c2h * lift * (us - uP);
    }
    sQ[k] = q;
  }
  __syncthreads();
  if (!active) return T(0);
  const int kk = le + 1, e = e0 + le;
  T r = T(0);
#pragma unroll
  for (int jn = 0; jn < NP1; ++jn) r += sD[n * NP1 + jn] * sQ[kk * NP1 + jn];
  r *= c2h;
  if (n == 0) {
    const T q0 = sQ[kk * NP1], qo = sQ[(kk - 1) * NP1 + P];
    const T qs = (a.dirichlet && e == 0) ? q0 : T(0.5) * (q0 + qo);
    r -= c2h * lift * (qs - q0);
  }
  if (n == P) {
    const T qP = sQ[kk * NP1 + P], qo = sQ[(kk + 1) * NP1];
    const T qs = (a.dirichlet && e == ne - 1) ? qP : T(0.5) * (qP + qo);
    r += c2h * lift * (qs - qP);
  }
  return cst<T>(a.kappa) * r;
}

// Extra shared memory of the 1D Burgers kernels (the viscous halo), in T units.
template <int DIM, int P, int EQ, int TK = 0>
__host__ __device__ constexpr int visc_smem_entries() {
  return (DIM == 1 && EQ == EXPDG_BURGERS) ? 2 * ((elems_per_block<1, P, TK>() + 2) * (P + 1) + 2) : 0;
}

// Shared-memory layout of the DG kernels (T units, then ints).
template <int DIM, int P, int EQ, typename T, int TK = 0>
struct DgSmem {
  static constexpr int NP1 = P + 1, NP = ipow(NP1, DIM), M = NFields<DIM, EQ>::value;
  static constexpr int SLOT = elems_per_block<DIM, P, TK>() * NP;
  __host__ __device__ static constexpr size_t bytes() {
    return sizeof(T) * ((size_t)DIM * M * SLOT + NP1 * NP1 + visc_smem_entries<DIM, P, EQ, TK>()) +
           sizeof(int) * elems_per_block<DIM, P, TK>() * 2 * DIM;
  }
  T* sF;    // [DIM][M][SLOT] fluxes
  T* sD;    // [NP1][NP1] derivative matrix
  T* sV;    // viscous halo (1D Burgers)
  int* sNb; // [EPB][2 DIM] neighbour elements
  __device__ explicit DgSmem(unsigned char* raw) {
    sF = reinterpret_cast<T*>(raw);
    sD = sF + DIM * M * SLOT;
    sV = sD + NP1 * NP1;
    sNb = reinterpret_cast<int*>(sV + visc_smem_entries<DIM, P, EQ, TK>());
  }
};

// One element group (the EPB elements from e0) of the DG operator; sD must
// hold the derivative matrix.  Every thread of the CTA calls it (it
// synchronises the CTA); trigger: signal dependent launches after the fluxes.
// It executes griddepcontrol.wait before its first read of memory another
// launch writes (after loading z when a.z_early).
// LINEAR = false: residual R(q), a.q = q.  LINEAR = true: linear operator,
// a.q = the linearisation state z of qt (k_linstate), a.v = v.
// T = double: FP64 (double in, double out); T = fx: float-float in, out
// float-float (a.out_h / a.out_l) or h + l in FP64 (a.out) (the residual of
// the FP32-operator forms: FP64-grade accuracy on the FP32 pipes);
// T = float: FP32 arithmetic on an FP32 input vector (linear operator), with
//   MX = false: float-float output (the float-float form);
//   MX = true:  the mixed form (FP64 Krylov basis): output in FP32 (a.out_h,
//               the operator's exact result) or widened exactly to FP64 on
//               the integer pipes (a.out); the augmentation tail in FP64.
template <int DIM, int P, int EQ, typename T, bool LINEAR, bool ROE, int TK = 0, bool MX = false>
__device__ __forceinline__ void dg_group(const DGArgs& a, const Tab& tab, int e0, const DgSmem<DIM, P, EQ, T, TK>& sm,
                                         bool trigger) {
  static_assert(!MX || (std::is_same<T, float>::value && LINEAR), "the mixed form's FP32 linear operator");
  constexpr int NP1 = P + 1;
  constexpr int NP = ipow(NP1, DIM);
  constexpr int M = NFields<DIM, EQ>::value;
  constexpr int EPB = elems_per_block<DIM, P, TK>();
  constexpr int SLOT = EPB * NP;  // nodes held by the CTA
  constexpr bool FF = !std::is_same<T, double>::value && !MX;  // float-float output
  using PH = Phys<DIM, EQ, T>;
  T* sF = sm.sF;
  const T* sD = sm.sD;
  T* sV = sm.sV;
  int* sNb = sm.sNb;

  const int tid = threadIdx.x;
  build_neighbours<DIM, P, TK>(a, e0, sNb);

  const int le = tid / NP;
  const int n = tid - le * NP;
  const int e = e0 + le;
  const bool active = (tid < SLOT) && (e < a.nelem);
  const T gamma = cst<T>(a.gamma);
  const T gm1 = gamma - T(1);
  const size_t stride = a.stride;
  const T* __restrict__ qin = static_cast<const T*>(a.q);
  const T* __restrict__ vin = static_cast<const T*>(a.v);
  T qv[M];  // residual: q at the node; linear: z at the node
  const bool early = LINEAR && a.z_early;
  if (early && active) {
    const size_t base = (size_t)e * NP + n;
#pragma unroll
    for (int f = 0; f < M; ++f) qv[f] = qin[f * stride + base];
  }
  griddep_wait();

  // Linear: the sub-step scalars (alpha, eta, the input's augmentation tail)
  // are read here, so their latency overlaps the operator's instead of
  // following it.  out = scale L v + sum_k cf_k W_{paug+1-k}.
  const bool aug = LINEAR && a.paug > 0 && (FF ? a.tail_h != nullptr : a.tail_d != nullptr);
  const bool dev = LINEAR && a.scal != nullptr;  // sub-step scalars in device memory
  double d_scale = a.alpha, d_cf[EXPDG_MAX_PHI];
  ff f_scale{a.alpha_h, a.alpha_l}, f_cf[EXPDG_MAX_PHI];
  float s_scale = a.alpha_h, s_cf[EXPDG_MAX_PHI];  // mixed form
  bool any = false;
  if constexpr (LINEAR) {
    if constexpr (MX) {
      // the tail entries narrowed on the integer pipes; eta is a power of two
      const float etaf = dev ? a.scal->eta_f : a.eta_f;
      if (dev) s_scale = a.scal->alpha_h;
#pragma unroll
      for (int k = 0; k < EXPDG_MAX_PHI; ++k) {
        s_cf[k] = (aug && k < a.paug) ? f64_to_f32_rn(a.tail_d[k]) * etaf : 0.0f;
        any |= (s_cf[k] != 0.0f);
      }
    } else if constexpr (!FF) {
      const double eta = dev ? a.scal->eta : a.eta;
      if (dev) d_scale = a.scal->alpha;
#pragma unroll
      for (int k = 0; k < EXPDG_MAX_PHI; ++k) {
        d_cf[k] = (aug && k < a.paug) ? eta * a.tail_d[k] : 0.0;
        any |= (d_cf[k] != 0.0);
      }
    } else {
      const float etaf = dev ? a.scal->eta_f : a.eta_f;
      if (dev) f_scale = ff{a.scal->alpha_h, a.scal->alpha_l};
#pragma unroll
      for (int k = 0; k < EXPDG_MAX_PHI; ++k) {
        f_cf[k] = ff{0.0f, 0.0f};
        if (aug && k < a.paug) f_cf[k] = ff{a.tail_h[k] * etaf, a.tail_l[k] * etaf};  // eta: a power of two
        any |= (f_cf[k].h != 0.0f);
      }
    }
  }

  T vv[M];  // linear: v at the node
  typename PH::Prim w{};
  T dp = T(0);
  if (active) {
    const size_t base = (size_t)e * NP + n;
#pragma unroll
    for (int f = 0; f < M; ++f) {
      if (!early) qv[f] = qin[f * stride + base];
      vv[f] = LINEAR ? vin[f * stride + base] : qv[f];
    }
    if (LINEAR) {
      dp = PH::lin_dp(qv, vv, gm1);
    } else {
      w = PH::prim(qv, gamma);
      if (!PH::physical(qv, w)) atomicOr(a.status, 1);
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      T F[M];
      if (LINEAR)
        PH::lin_flux(qv, vv, dp, d, F);
      else
        PH::flux(qv, w, d, F);
#pragma unroll
      for (int f = 0; f < M; ++f) sF[(d * M + f) * SLOT + tid] = F[f];
    }
  }
  __syncthreads();
  if (trigger) griddep_launch();
  T visc = T(0);
  if constexpr (DIM == 1 && EQ == EXPDG_BURGERS) {
    constexpr int NH2 = visc_smem_entries<DIM, P, EQ, TK>() / 2;
    if (a.viscous) {  // uniform
      if constexpr (LINEAR)
        visc = visc_term<P, T, TK>(a, vin, sD, cst<T>(tab.lift), sV, sV + NH2, e0, tid, le, n, active);
      else
        visc = visc_term<P, T, TK>(a, qin, sD, cst<T>(tab.lift), sV, sV + NH2, e0, tid, le, n, active);
    }
  }
  if (!active) return;  // no further synchronisation below

  T acc[M];
  node_terms<DIM, P, EQ, T, LINEAR, ROE, TK>(
      a, cst<T>(tab.lift), [&](int f, size_t gi) { return qin[f * stride + gi]; }, sF, sD, sNb, tid, le, n, qv, vv,
      w, [&](int f, size_t gi) { return vin[f * stride + gi]; }, acc);
  acc[0] += visc;

  const size_t base = (size_t)e * NP + n;
  if constexpr (std::is_same<T, fx>::value) {  // residual in float-float: out = alpha (R + s)
    static_assert(!LINEAR, "the float-float kernels compute the residual");
    const fx al(a.alpha_h, a.alpha_l);
    const bool wide = a.out != nullptr;  // uniform: FP64 output (mixed form)
#pragma unroll
    for (int f = 0; f < M; ++f) {
      fx o = al * acc[f];
      if (a.src != nullptr) o = o + fx(a.alpha * a.src[f * stride + base]);
      if (wide) {  // h + l: at most 48 significant bits, exact in binary64
        a.out[f * stride + base] = f32_to_f64_exact(o.h) + f32_to_f64_exact(o.l);
      } else {
        a.out_h[f * stride + base] = o.h;
        a.out_l[f * stride + base] = o.l;
      }
    }
    return;
  } else if constexpr (MX) {  // FP32 arithmetic to the end
    const bool wide = a.out != nullptr;  // uniform
#pragma unroll
    for (int f = 0; f < M; ++f) {
      const size_t gi = f * stride + base;
      float o = acc[f] * s_scale;
      if (any) {
#pragma unroll
        for (int k = 1; k <= EXPDG_MAX_PHI; ++k)
          if (k <= a.paug && s_cf[k - 1] != 0.0f) o = fmaf(s_cf[k - 1], a.W_f[a.paug + 1 - k][gi], o);
      }
      if (wide)
        a.out[gi] = f32_to_f64_exact(o);
      else
        a.out_h[gi] = o;
    }
    if (aug && e0 == 0 && tid == 0)
      for (int k = 0; k < a.paug; ++k) a.out_tail_d[k] = (k + 1 < a.paug) ? a.tail_d[k + 1] : 0.0;
    return;
  } else if constexpr (!FF) {
    const double scale = d_scale;
    const double* cf = d_cf;
#pragma unroll
    for (int f = 0; f < M; ++f) {
      double o = scale * (double)acc[f];
      if (!LINEAR && a.src != nullptr) o += a.alpha * a.src[f * stride + base];
      if (any) {
        const size_t gi = f * stride + base;
#pragma unroll
        for (int k = 1; k <= EXPDG_MAX_PHI; ++k)
          if (k <= a.paug && cf[k - 1] != 0.0) o += cf[k - 1] * a.W_d[a.paug + 1 - k][gi];
      }
      a.out[f * stride + base] = o;
    }
    if (aug && e0 == 0 && tid == 0)
      for (int k = 0; k < a.paug; ++k) a.out_tail_d[k] = (k + 1 < a.paug) ? a.tail_d[k + 1] : 0.0;
  } else {
    const ff scale = f_scale;
    const ff* cf = f_cf;
#pragma unroll
    for (int f = 0; f < M; ++f) {
      // exact float * float-float product, then the augmentation in float-float
      float p = __fmul_rn((float)acc[f], scale.h);
      float pe = __fmaf_rn((float)acc[f], scale.h, -p);
      pe = __fmaf_rn((float)acc[f], scale.l, pe);
      ff o = ff_fast_two_sum(p, pe);
      if (!LINEAR && a.src != nullptr) o = ff_add(o, ff_from_double(a.alpha * a.src[f * stride + base]));
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
    if (aug && e0 == 0 && tid == 0)
      for (int k = 0; k < a.paug; ++k) {
        const ff t = (k + 1 < a.paug) ? ff{a.tail_h[k + 1], a.tail_l[k + 1]} : ff{0.0f, 0.0f};
        a.out_tail_h[k] = t.h;
        a.out_tail_l[k] = t.l;
      }
  }
}

template <int DIM, int P, int EQ, typename T, bool LINEAR, bool ROE, int TK, bool MX>
__global__ void __launch_bounds__(dg_threads<DIM, P, TK>())
k_dg(const DGArgs a, const Tab tab) {
  // the tables and the neighbour lists come from the parameters: set up before
  // the wait (dg_group waits)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const DgSmem<DIM, P, EQ, T, TK> sm(smem_raw);
  for (int k = threadIdx.x; k < (P + 1) * (P + 1); k += blockDim.x) sm.sD[k] = d_entry<T>(tab, k);
  dg_group<DIM, P, EQ, T, LINEAR, ROE, TK, MX>(a, tab, blockIdx.x * elems_per_block<DIM, P, TK>(), sm, true);
}

template <int DIM, int P, int EQ, typename T, bool LINEAR, bool ROE, int TK = 0, bool MX = false>
cudaError_t launch_dg_t(const DGArgs& a, const Tab& t, cudaStream_t s) {
  constexpr int EPB = elems_per_block<DIM, P, TK>();
  const int threads = dg_threads<DIM, P, TK>();
  const size_t smem = DgSmem<DIM, P, EQ, T, TK>::bytes();
  const int blocks = (a.nelem + EPB - 1) / EPB;
  auto kern = k_dg<DIM, P, EQ, T, LINEAR, ROE, TK, MX>;
  // once per instantiation, thread-safe (function-local static initialisation)
  static const cudaError_t configured =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (configured != cudaSuccess) return configured;
  if (blocks == 0) return cudaSuccess;
  return pdl_launch(kern, dim3(blocks), dim3(threads), smem, s, a, t);
}

// The FP32 operator apply in the tile class a.tile (0, 1, 2: CTAs of about
// 256, 128, 512 threads); the other kernels use class 0.
template <int DIM, int P, int EQ, typename T, bool LINEAR, bool ROE, bool MX>
cudaError_t launch_dg_tile(const DGArgs& a, const Tab& t, cudaStream_t s) {
  if constexpr (LINEAR && std::is_same<T, float>::value) {
    if (a.tile == 1) return launch_dg_t<DIM, P, EQ, T, LINEAR, ROE, 1, MX>(a, t, s);
    if (a.tile == 2) return launch_dg_t<DIM, P, EQ, T, LINEAR, ROE, 2, MX>(a, t, s);
  }
  return launch_dg_t<DIM, P, EQ, T, LINEAR, ROE, 0, MX>(a, t, s);
}

template <int DIM, int EQ, typename T, bool LINEAR, bool ROE, bool MX = false>
cudaError_t launch_dg_p(int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  switch (p) {
    case 1: return launch_dg_tile<DIM, 1, EQ, T, LINEAR, ROE, MX>(a, t, s);
    case 2: return launch_dg_tile<DIM, 2, EQ, T, LINEAR, ROE, MX>(a, t, s);
    case 3: return launch_dg_tile<DIM, 3, EQ, T, LINEAR, ROE, MX>(a, t, s);
    case 4: return launch_dg_tile<DIM, 4, EQ, T, LINEAR, ROE, MX>(a, t, s);
    case 5: return launch_dg_tile<DIM, 5, EQ, T, LINEAR, ROE, MX>(a, t, s);
    case 6: return launch_dg_tile<DIM, 6, EQ, T, LINEAR, ROE, MX>(a, t, s);
    case 7: return launch_dg_tile<DIM, 7, EQ, T, LINEAR, ROE, MX>(a, t, s);
    case 8: return launch_dg_tile<DIM, 8, EQ, T, LINEAR, ROE, MX>(a, t, s);
    default: return cudaErrorInvalidValue;
  }
}

// Float-float residual (the float-float form's R).
template <int DIM, int EQ, bool ROE = false>
cudaError_t launch_dg_fx_dim(int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  return launch_dg_p<DIM, EQ, fx, false, ROE>(p, a, t, s);
}

}  // namespace expdg
