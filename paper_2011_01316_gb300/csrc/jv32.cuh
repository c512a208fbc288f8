// The FP32 linear operator L(qt) v of the 2D and 3D Euler equations (the
// mixed and float-float forms' Jv; paper Sec. 2.2 Eq. linearflux, Sec. 3.2
// (A~q)*, LF coefficient of Sec. 5.1 or the Roe matrix of Sec. 3.2, frozen
// at the linearisation state).  Same operator as k_dg<..., float, LINEAR>,
// organised for fewer instructions per node:
//
//   - per-node data are packed for vector shared-memory accesses: a node's
//     fields 0..3 as one float4 (and field 4 of 3D as a float) for the
//     fluxes of each direction, for the linearisation state z and for the
//     input v, so the derivative reads a line's fluxes with one 16-byte load
//     per node and accumulates two fields per packed FMA (FFMA2);
//   - a face whose neighbour element lies in the same CTA (the elements of a
//     CTA are consecutive along x, so most x faces) takes the neighbour's
//     flux, z and v from shared memory instead of re-loading them and
//     re-forming the flux;
//   - the per-field base pointers are formed once and the node indices are
//     32-bit.
//
// Every rounding is written with the _rn intrinsics, which the compiler never
// contracts or reorders: a flux formed by its own node's thread and the same
// flux re-formed by a thread of the neighbouring CTA agree bit for bit, so
// the result does not depend on the tile class (which faces are internal).
#pragma once

#include "dg_impl.cuh"

namespace expdg {
namespace jv32 {

// Fields of a node as a float4 (fields 0..3) and, for 3D, a fifth float.
template <int M>
struct NodeV {
  float4 a;
  float b;  // field 4 (3D only)
  __device__ __forceinline__ float get(int f) const {
    return f == 0 ? a.x : f == 1 ? a.y : f == 2 ? a.z : f == 3 ? a.w : b;
  }
};

__device__ __forceinline__ float2 lo(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi(float4 v) { return make_float2(v.z, v.w); }

// Pressure perturbation dp = (gamma - 1)(v_E - u.v_m + |u|^2 v_rho / 2) at z.
template <int DIM>
__device__ __forceinline__ float lin_dp(const NodeV<DIM + 2>& z, const NodeV<DIM + 2>& v, float gm1) {
  float uu = __fmul_rn(z.get(0), z.get(0)), uv = __fmul_rn(z.get(0), v.get(1));
#pragma unroll
  for (int k = 1; k < DIM; ++k) {
    uu = __fmaf_rn(z.get(k), z.get(k), uu);
    uv = __fmaf_rn(z.get(k), v.get(1 + k), uv);
  }
  const float t = __fmaf_rn(__fmul_rn(0.5f, uu), v.get(0), __fsub_rn(v.get(DIM + 1), uv));
  return __fmul_rn(gm1, t);
}

// A_d(qt) v = (v_md, v_mk u_d + u_k du + delta_kd dp, (v_E + dp) u_d + H du),
// du = v_md - u_d v_rho, from z = (u, H, a) (or (u, H, sqrt(rho)) for Roe).
template <int DIM>
__device__ __forceinline__ NodeV<DIM + 2> lin_flux(const NodeV<DIM + 2>& z, const NodeV<DIM + 2>& v, float dp,
                                                    int d) {
  const float ud = z.get(d);
  const float du = __fmaf_rn(-ud, v.get(0), v.get(1 + d));
  float F[DIM + 2];
  F[0] = v.get(1 + d);
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    float t = __fmaf_rn(z.get(k), du, __fmul_rn(v.get(1 + k), ud));
    if (k == d) t = __fadd_rn(t, dp);
    F[1 + k] = t;
  }
  F[DIM + 1] = __fmaf_rn(z.get(DIM), du, __fmul_rn(__fadd_rn(v.get(DIM + 1), dp), ud));
  NodeV<DIM + 2> out;
  out.a = make_float4(F[0], F[1], F[2], F[3]);
  out.b = (DIM == 3) ? F[4] : 0.0f;
  return out;
}

template <int DIM, int P, int TK, int TC = 0>
struct Smem {
  static constexpr int NP1 = P + 1, NP = ipow(NP1, DIM), EPB = elems_per_block<DIM, P, TK>(), SLOT = EPB * NP;
  static constexpr bool F5 = DIM == 3;  // a fifth field
  __host__ __device__ static constexpr size_t bytes() {
    return sizeof(float4) * ((size_t)DIM * SLOT + 2 * SLOT) +  // fluxes, z, v (fields 0..3)
           (F5 ? sizeof(float) * (size_t)DIM * SLOT + sizeof(float2) * SLOT : 0) +  // field 4
           sizeof(float) * NP1 * NP1 + sizeof(int) * EPB * 2 * DIM +
           (TC ? sizeof(float) * (size_t)DIM * (DIM + 2) * SLOT : 0);  // tensor-core derivatives
  }
  float4* F4;  // [DIM][SLOT]
  float4* Z4;  // [SLOT]
  float4* V4;  // [SLOT]
  float* F1;   // [DIM][SLOT] (3D)
  float2* ZV1; // [SLOT] (z_4, v_4) (3D)
  float* D;    // [NP1][NP1]
  int* Nb;     // [EPB][2 DIM]
  float* Der;  // [DIM][M][SLOT] derivatives formed on the tensor cores (TC)
  __device__ explicit Smem(unsigned char* raw) {
    F4 = reinterpret_cast<float4*>(raw);
    Z4 = F4 + DIM * SLOT;
    V4 = Z4 + SLOT;
    unsigned char* p = reinterpret_cast<unsigned char*>(V4 + SLOT);
    if (F5) {
      ZV1 = reinterpret_cast<float2*>(p);
      F1 = reinterpret_cast<float*>(ZV1 + SLOT);
      p = reinterpret_cast<unsigned char*>(F1 + DIM * SLOT);
    } else {
      ZV1 = nullptr;
      F1 = nullptr;
    }
    D = reinterpret_cast<float*>(p);
    Nb = reinterpret_cast<int*>(D + NP1 * NP1);
    Der = reinterpret_cast<float*>(Nb + EPB * 2 * DIM);
  }
};

// ---- the derivative contraction on the tensor cores (experiment K7) ----
// TF32 bits of x, rounded to nearest (ties away).
__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// c += a b for one m16n8k8 TF32 tile (warp-wide; FP32 accumulation).
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// All derivatives sum_j D(i, j) F_d(line node j) of the CTA's fluxes as
// matrix products on the tensor cores, into Der: for each direction d and
// field f, the lines along x_d are the rows of A (16 lines per tile, their
// P+1 nodes the K dimension, padded to multiples of 8 with zeros) and
// B = D^T (K x N, N = P+1 output nodes, padded likewise); warp-level
// m16n8k8 TF32 MMAs with FP32 accumulation.  TC = 1: one TF32 product
// (operands rounded to 10-bit significands); TC = 3: the split x = hi + lo
// of both operands and three products (lo hi + hi lo + hi hi, about FP32
// accuracy).  Every thread of the CTA calls it; it ends with a barrier.
template <int DIM, int P, int TK, int TC>
__device__ __forceinline__ void tc_derivative(const Smem<DIM, P, TK, TC>& sm, int tid) {
  constexpr int M = DIM + 2, NP1 = P + 1, NP = ipow(NP1, DIM), EPB = elems_per_block<DIM, P, TK>(),
                SLOT = EPB * NP;
  constexpr int LPE = ipow(NP1, DIM - 1), L = EPB * LPE, NG = (L + 15) / 16, KS = (NP1 + 7) / 8;
  const int lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  uint32_t bh[KS][KS][2], bl[KS][KS][2];  // [k step][n tile][2]: B(k, n) = D(n, k)
#pragma unroll
  for (int ks = 0; ks < KS; ++ks)
#pragma unroll
    for (int nt = 0; nt < KS; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = t4 + 4 * h + 8 * ks, nn = g + 8 * nt;
        const float x = (k < NP1 && nn < NP1) ? sm.D[nn * NP1 + k] : 0.0f;
        bh[ks][nt][h] = tf32_of(x);
        bl[ks][nt][h] = tf32_of(__fsub_rn(x, __uint_as_float(bh[ks][nt][h])));
      }
  for (int task = warp; task < DIM * M * NG; task += nwarp) {  // warp-uniform
    const int d = task / (M * NG), f = (task / NG) % M, grp = task % NG;
    const int sd = (d == 0) ? 1 : (d == 1 ? NP1 : NP1 * NP1);
    // this thread's two rows (lines) g and g + 8 of the tile: their first slots
    int st[2];
    bool ok[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = grp * 16 + g + 8 * h;
      ok[h] = r < L;
      const int le = ok[h] ? r / LPE : 0, l = ok[h] ? r - (r / LPE) * LPE : 0;
      int o;
      if (d == 0)
        o = NP1 * l;
      else if (d == 1)
        o = (l % NP1) + NP1 * NP1 * (l / NP1);
      else
        o = l;
      st[h] = le * NP + o;
    }
    const float* Fd = (f < 4) ? reinterpret_cast<const float*>(sm.F4 + d * SLOT) + f : sm.F1 + d * SLOT;
    const int fs = (f < 4) ? 4 : 1;
    float c[KS][4];
#pragma unroll
    for (int nt = 0; nt < KS; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      float av[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {  // a0: (g, t4), a1: (g + 8, t4), a2: (g, t4 + 4), a3: (g + 8, t4 + 4)
        const int h = q & 1, k = t4 + 4 * (q >> 1) + 8 * ks;
        av[q] = (ok[h] && k < NP1) ? Fd[(st[h] + k * sd) * fs] : 0.0f;
      }
      uint32_t ah[4], al[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ah[q] = tf32_of(av[q]);
        al[q] = tf32_of(__fsub_rn(av[q], __uint_as_float(ah[q])));
      }
#pragma unroll
      for (int nt = 0; nt < KS; ++nt) {
        if (TC == 3) {
          mma_tf32(c[nt], al, bh[ks][nt]);
          mma_tf32(c[nt], ah, bl[ks][nt]);
        }
        mma_tf32(c[nt], ah, bh[ks][nt]);
      }
    }
    float* out = sm.Der + (d * M + f) * SLOT;
#pragma unroll
    for (int nt = 0; nt < KS; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {  // c0: (g, 2 t4), c1: (g, 2 t4 + 1), c2: (g + 8, 2 t4), c3: (g + 8, 2 t4 + 1)
        const int h = q >> 1, nn = 2 * t4 + (q & 1) + 8 * nt;
        if (ok[h] && nn < NP1) out[st[h] + nn * sd] = c[nt][q];
      }
  }
  __syncthreads();
}

}  // namespace jv32

// MX = true: the mixed form's output (FP32 to a.out_h, or widened to FP64 in
// a.out; FP64 augmentation tail); false: the float-float form's (float-float
// output and tail).
// TC (experiment K7): 0 the derivative in FP32 on the FMA pipes; 1 or 3 on the
// tensor cores (tc_derivative).  LF: at most 32 registers (a full SM of
// resident threads: the kernel is latency bound); Roe keeps more state live.
template <int DIM, int P, bool ROE, int TK, bool MX, int TC = 0>
__global__ void __launch_bounds__(dg_threads<DIM, P, TK>(), (ROE || TC) ? 1 : 2048 / dg_threads<DIM, P, TK>())
    k_jv32(const DGArgs a, const Tab tab) {
  using namespace jv32;
  constexpr int M = DIM + 2, NP1 = P + 1, NP = ipow(NP1, DIM), NF = 2 * DIM;
  constexpr int EPB = elems_per_block<DIM, P, TK>(), SLOT = EPB * NP;
  using SM = Smem<DIM, P, TK, TC>;
  using NV = NodeV<M>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SM sm(smem_raw);
  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * EPB;
  // tables and neighbour lists come from the parameters: before the wait
  for (int k = tid; k < NP1 * NP1; k += blockDim.x) sm.D[k] = tab.Dh[k];
  build_neighbours<DIM, P, TK>(a, e0, sm.Nb);

  const int le = tid / NP, n = tid - le * NP, e = e0 + le;
  const bool active = (tid < SLOT) && (e < a.nelem);
  const unsigned stride = (unsigned)a.stride;
  const float* __restrict__ zin = static_cast<const float*>(a.q);
  const float* __restrict__ vin = static_cast<const float*>(a.v);
  const unsigned base = (unsigned)e * NP + n;
  auto load = [&](const float* __restrict__ p, unsigned i) {
    NV x;
    x.a = make_float4(p[i], p[i + stride], p[i + 2 * stride], p[i + 3 * stride]);
    x.b = (DIM == 3) ? p[i + 4 * stride] : 0.0f;
    return x;
  };
  NV z{}, v{};
  // z was written by a launch that completed before this launch's predecessor
  // started (inside an Arnoldi step): read it before the wait
  if (a.z_early && active) z = load(zin, base);
  griddep_wait();
  if (!a.z_early && active) z = load(zin, base);

  // sub-step scalars: out = scale L v + sum_k cf_k W_{paug+1-k}
  const bool aug = a.paug > 0 && (MX ? a.tail_d != nullptr : a.tail_h != nullptr);
  const bool dev = a.scal != nullptr;
  float s_scale = a.alpha_h, s_cf[EXPDG_MAX_PHI];
  ff f_scale{a.alpha_h, a.alpha_l}, f_cf[EXPDG_MAX_PHI];
  bool any = false;
  {
    const float etaf = dev ? a.scal->eta_f : a.eta_f;
    if (dev) {
      s_scale = a.scal->alpha_h;
      f_scale = ff{a.scal->alpha_h, a.scal->alpha_l};
    }
#pragma unroll
    for (int k = 0; k < EXPDG_MAX_PHI; ++k) {
      s_cf[k] = 0.0f;
      f_cf[k] = ff{0.0f, 0.0f};
      if (aug && k < a.paug) {
        if constexpr (MX)
          s_cf[k] = __fmul_rn(f64_to_f32_rn(a.tail_d[k]), etaf);  // eta: a power of two
        else
          f_cf[k] = ff{a.tail_h[k] * etaf, a.tail_l[k] * etaf};
      }
      any |= MX ? (s_cf[k] != 0.0f) : (f_cf[k].h != 0.0f);
    }
  }

  const float gm1 = __fsub_rn(a.gamma.h, 1.0f);
  if (active) {
    v = load(vin, base);
    const float dp = lin_dp<DIM>(z, v, gm1);
    sm.Z4[tid] = z.a;
    sm.V4[tid] = v.a;
    if (DIM == 3) sm.ZV1[tid] = make_float2(z.b, v.b);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const NV F = lin_flux<DIM>(z, v, dp, d);
      sm.F4[d * SLOT + tid] = F.a;
      if (DIM == 3) sm.F1[d * SLOT + tid] = F.b;
    }
  }
  __syncthreads();
  griddep_launch();
  if constexpr (TC != 0) tc_derivative<DIM, P, TK, TC>(sm, tid);
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
  const float lift = tab.lift.h;
  float2 acc01 = make_float2(0.f, 0.f), acc23 = make_float2(0.f, 0.f);
  float acc4 = 0.0f;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int sd = (d == 0) ? 1 : (d == 1 ? NP1 : NP1 * NP1);
    const float c2h = a.two_over_h[d].h;
    const int lbase = tid - ii[d] * sd;
    // derivative along x_d: sum_j D(i_d, j) F_d(line node j), two fields per packed FMA
    float2 s01 = make_float2(0.f, 0.f), s23 = make_float2(0.f, 0.f);
    float s4 = 0.0f;
    if constexpr (TC != 0) {
      const float* Dd = sm.Der + d * M * SLOT + tid;
      s01 = make_float2(Dd[0], Dd[SLOT]);
      s23 = make_float2(Dd[2 * SLOT], Dd[3 * SLOT]);
      if (DIM == 3) s4 = Dd[4 * SLOT];
    } else {
#pragma unroll
      for (int j = 0; j < NP1; ++j) {
        const float dj = sm.D[ii[d] * NP1 + j];
        const float2 dd = make_float2(dj, dj);
        const float4 F = sm.F4[d * SLOT + lbase + j * sd];
        s01 = __ffma2_rn(dd, lo(F), s01);
        s23 = __ffma2_rn(dd, hi(F), s23);
        if (DIM == 3) s4 = __fmaf_rn(dj, sm.F1[d * SLOT + lbase + j * sd], s4);
      }
    }
    const float2 mc = make_float2(-c2h, -c2h);
    acc01 = __ffma2_rn(mc, s01, acc01);
    acc23 = __ffma2_rn(mc, s23, acc23);
    if (DIM == 3) acc4 = __fmaf_rn(-c2h, s4, acc4);
    // face term: -(2/h_d)(1/w_0)(F*.n - F^-.n) with
    // F*.n - F^-.n = 1/2 [sgn (F^+ - F^-) + D (v^- - v^+)], D = lambda (LF) or |A(q*_Roe)|
    if (ii[d] == 0 || ii[d] == P) {
      const bool up = ii[d] == P;
      const int en = sm.Nb[le * NF + 2 * d + (up ? 1 : 0)];
      const int nn = n + (up ? -P : P) * sd;
      const int ls = (en - e0) * NP + nn;  // the neighbour node's slot if its element is in the CTA
      const bool inside = en >= e0 && en < e0 + EPB && en < a.nelem;
      NV zn, vn, Fp;
      if (inside) {
        zn.a = sm.Z4[ls];
        vn.a = sm.V4[ls];
        Fp.a = sm.F4[d * SLOT + ls];
        if (DIM == 3) {
          const float2 t = sm.ZV1[ls];
          zn.b = t.x;
          vn.b = t.y;
          Fp.b = sm.F1[d * SLOT + ls];
        }
      } else {
        const unsigned nb = (unsigned)en * NP + nn;
        zn = load(zin, nb);
        vn = load(vin, nb);
        Fp = lin_flux<DIM>(zn, vn, lin_dp<DIM>(zn, vn, gm1), d);
      }
      // the node's own flux, z and v from shared memory (not kept in
      // registers across the barrier: fewer registers, more resident warps)
      NV Fm, zo, vo;
      Fm.a = sm.F4[d * SLOT + tid];
      Fm.b = (DIM == 3) ? sm.F1[d * SLOT + tid] : 0.0f;
      zo.a = sm.Z4[tid];
      vo.a = sm.V4[tid];
      if (DIM == 3) {
        const float2 t = sm.ZV1[tid];
        zo.b = t.x;
        vo.b = t.y;
      }
      // jump of the flux, oriented by the outward normal
      float jF[M], dq[M];
#pragma unroll
      for (int f = 0; f < M; ++f) {
        jF[f] = up ? __fsub_rn(Fp.get(f), Fm.get(f)) : __fsub_rn(Fm.get(f), Fp.get(f));
        dq[f] = __fsub_rn(vo.get(f), vn.get(f));
      }
      float Dq[M];
      if constexpr (ROE) {  // z = (u, H, sqrt(rho)) on both sides
        float zm[M], zp[M];
#pragma unroll
        for (int f = 0; f < M; ++f) {
          zm[f] = zo.get(f);
          zp[f] = zn.get(f);
        }
        Phys<DIM, EXPDG_EULER, float>::roe_dissipation(zm, zm[M - 2], zm[M - 1], zp, zp[M - 2], zp[M - 1], dq, d,
                                                       gm1, Dq);
      } else {
        const float lam =
            fmaxf(__fadd_rn(fabsf(zo.get(d)), zo.get(DIM + 1)), __fadd_rn(fabsf(zn.get(d)), zn.get(DIM + 1)));
#pragma unroll
        for (int f = 0; f < M; ++f) Dq[f] = __fmul_rn(lam, dq[f]);
      }
      const float k = __fmul_rn(__fmul_rn(c2h, lift), -0.5f);
      const float2 kk = make_float2(k, k);
      acc01 = __ffma2_rn(kk, __fadd2_rn(make_float2(jF[0], jF[1]), make_float2(Dq[0], Dq[1])), acc01);
      acc23 = __ffma2_rn(kk, __fadd2_rn(make_float2(jF[2], jF[3]), make_float2(Dq[2], Dq[3])), acc23);
      if (DIM == 3) acc4 = __fmaf_rn(k, __fadd_rn(jF[4], Dq[4]), acc4);
    }
  }

  const float acc[5] = {acc01.x, acc01.y, acc23.x, acc23.y, acc4};
  if constexpr (MX) {
    const bool wide = a.out != nullptr;  // uniform
#pragma unroll
    for (int f = 0; f < M; ++f) {
      const unsigned gi = base + f * stride;
      float o = __fmul_rn(acc[f], s_scale);
      if (any) {
#pragma unroll
        for (int k = 1; k <= EXPDG_MAX_PHI; ++k)
          if (k <= a.paug && s_cf[k - 1] != 0.0f) o = __fmaf_rn(s_cf[k - 1], a.W_f[a.paug + 1 - k][gi], o);
      }
      if (wide)
        a.out[gi] = f32_to_f64_exact(o);
      else
        a.out_h[gi] = o;
    }
    if (aug && e0 == 0 && tid == 0)
      for (int k = 0; k < a.paug; ++k) a.out_tail_d[k] = (k + 1 < a.paug) ? a.tail_d[k + 1] : 0.0;
  } else {
#pragma unroll
    for (int f = 0; f < M; ++f) {
      const unsigned gi = base + f * stride;
      // exact float * float-float product, then the augmentation in float-float
      const float p = __fmul_rn(acc[f], f_scale.h);
      float pe = __fmaf_rn(acc[f], f_scale.h, -p);
      pe = __fmaf_rn(acc[f], f_scale.l, pe);
      ff o = ff_fast_two_sum(p, pe);
      if (any) {
#pragma unroll
        for (int k = 1; k <= EXPDG_MAX_PHI; ++k)
          if (k <= a.paug && f_cf[k - 1].h != 0.0f) {
            const int wi = a.paug + 1 - k;
            o = ff_fma(f_cf[k - 1], ff{a.W_h[wi][gi], a.W_l[wi][gi]}, o);
          }
      }
      a.out_h[gi] = o.h;
      a.out_l[gi] = o.l;
    }
    if (aug && e0 == 0 && tid == 0)
      for (int k = 0; k < a.paug; ++k) {
        const ff t = (k + 1 < a.paug) ? ff{a.tail_h[k + 1], a.tail_l[k + 1]} : ff{0.0f, 0.0f};
        a.out_tail_h[k] = t.h;
        a.out_tail_l[k] = t.l;
      }
  }
}

template <int DIM, int P, bool ROE, int TK, bool MX, int TC = 0>
cudaError_t launch_jv32_t(const DGArgs& a, const Tab& t, cudaStream_t s) {
  constexpr int EPB = elems_per_block<DIM, P, TK>();
  const int threads = dg_threads<DIM, P, TK>();
  const size_t smem = jv32::Smem<DIM, P, TK, TC>::bytes();
  const int blocks = (a.nelem + EPB - 1) / EPB;
  auto kern = k_jv32<DIM, P, ROE, TK, MX, TC>;
  static const cudaError_t configured =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (configured != cudaSuccess) return configured;
  if (blocks == 0) return cudaSuccess;
  return pdl_launch(kern, dim3(blocks), dim3(threads), smem, s, a, t);
}

// tile classes 0..2: CTA sizes; 3 and 4 (the LF mixed form): the 256-thread
// CTA with the derivative on the tensor cores, 3xTF32 and TF32 (experiment K7)
template <int DIM, int P, bool ROE, bool MX>
cudaError_t launch_jv32_tile(const DGArgs& a, const Tab& t, cudaStream_t s) {
  if (a.tile == 1) return launch_jv32_t<DIM, P, ROE, 1, MX>(a, t, s);
  if (a.tile == 2) return launch_jv32_t<DIM, P, ROE, 2, MX>(a, t, s);
  if constexpr (MX && !ROE) {
    if (a.tile == 3) return launch_jv32_t<DIM, P, ROE, 0, MX, 3>(a, t, s);
    if (a.tile == 4) return launch_jv32_t<DIM, P, ROE, 0, MX, 1>(a, t, s);
  }
  return launch_jv32_t<DIM, P, ROE, 0, MX>(a, t, s);
}

// The FP32 linear operator of 2D / 3D Euler in the mixed (MX) or float-float form.
template <int DIM, bool ROE, bool MX>
cudaError_t launch_jv32(int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  switch (p) {
    case 1: return launch_jv32_tile<DIM, 1, ROE, MX>(a, t, s);
    case 2: return launch_jv32_tile<DIM, 2, ROE, MX>(a, t, s);
    case 3: return launch_jv32_tile<DIM, 3, ROE, MX>(a, t, s);
    case 4: return launch_jv32_tile<DIM, 4, ROE, MX>(a, t, s);
    case 5: return launch_jv32_tile<DIM, 5, ROE, MX>(a, t, s);
    case 6: return launch_jv32_tile<DIM, 6, ROE, MX>(a, t, s);
    case 7: return launch_jv32_tile<DIM, 7, ROE, MX>(a, t, s);
    case 8: return launch_jv32_tile<DIM, 8, ROE, MX>(a, t, s);
    default: return cudaErrorInvalidValue;
  }
}

// form: DG_F64, or (linear operator only) DG_F32_FF or DG_F32_MX.  The FP32
// linear operator of 2D / 3D Euler runs k_jv32 when its 32-bit node indices
// cover the arrays (fields x unknowns per field < 2^32), else k_dg.
// ROE: the Roe-flux instantiations (Euler), built in their own translation units.
template <int DIM, int EQ, bool ROE = false>
cudaError_t launch_dg_dim(bool linear, int form, int p, const DGArgs& a, const Tab& t, cudaStream_t s) {
  constexpr bool JV32 = DIM >= 2 && EQ == EXPDG_EULER;
  const bool fits = (size_t)(DIM + 2) * a.stride < ((size_t)1 << 32);
  if (form == DG_F32_MX) {
    if (!linear) return cudaErrorInvalidValue;
    if constexpr (JV32)
      if (fits) return launch_jv32<DIM, ROE, true>(p, a, t, s);
    return launch_dg_p<DIM, EQ, float, true, ROE, true>(p, a, t, s);
  }
  if (form == DG_F32_FF) {
    if (!linear) return cudaErrorInvalidValue;
    if constexpr (JV32)
      if (fits) return launch_jv32<DIM, ROE, false>(p, a, t, s);
    return launch_dg_p<DIM, EQ, float, true, ROE>(p, a, t, s);
  }
  return linear ? launch_dg_p<DIM, EQ, double, true, ROE>(p, a, t, s)
                : launch_dg_p<DIM, EQ, double, false, ROE>(p, a, t, s);
}

}  // namespace expdg
