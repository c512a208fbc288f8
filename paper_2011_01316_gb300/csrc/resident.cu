// CTA-resident EPI2 solves: one launch advances a whole class of small
// instances (same equation, dimension, order and arithmetic form; any mesh
// size, step size, tolerance and window), one CTA per instance, every step of
// every instance inside the launch.
//
// A small instance run through the streaming path pays a chain of about
// three launches per Arnoldi step and a host read-back per error check; here
// the chain is a CTA barrier and the check is taken on the device.  Each CTA
// runs the method as the paper defines it (Sec. 2.3 with the Krylov reading
// the CPU oracle takes decision for decision):
//
//   per step:   z = linearisation state of q^n, r = dt R(q^n);
//               w = phi_1(dt L) r by the augmented Krylov method with
//               A_hat = [[dt L, eta r], [0, 0]], start [0; 1/eta];
//               q^{n+1} = q^n + w                      (EPI2, Sec. 5.1)
//   Krylov:     modified Gram-Schmidt over the window (iop > 0) or over all
//               earlier vectors (iop = 0); checks at m = m_step, 2 m_step,
//               ..., m_max with Saad's estimate beta h_{m+1,m} |e_m^T
//               exp(H_m) e_1| <= tol beta; happy breakdown when h_{m+1,m}
//               <= 1e-13 ||A_hat v_m||; on reaching m_max the sub-step
//               halves, after an accepted sub-step with m <= m_max / 2 it
//               doubles (never past the end), the sub-step vectors from the
//               paper's recurrence (Sec. 2.3: chat_0 = w(s), chat_1 = c_1);
//               eta = 2^-round(log2 ||sigma c_1||).
//   exp(H_m):   scaling to ||H / 2^s||_1 <= 1/2, Taylor degree 18 by
//               Horner, s squarings (Moler & Van Loan's method 3).
//
// Arithmetic forms: FP64 throughout; or the mixed form (the linear operator
// in FP32 on the FP32 rounding of each basis vector, with FP32
// accumulation; the residual in float-float; the Krylov basis, inner
// products, orthogonalisation, exp(H_m) and the update in FP64).
//
// The DG operators are the streaming kernels' element-group code (dg_group),
// run over the instance's element groups in turn; every vector pass loops
// over the instance's unknowns with the CTA's threads; every sum has a fixed
// order, so an instance gives the same bits alone or in any batch.
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "dg_impl.cuh"
#include "tables.h"

namespace expdg {

namespace {

constexpr int RES_MMAX = EXPDG_BATCH_MAX_KRYLOV;  // Krylov dimension limit of a resident solve
constexpr int HC = RES_MMAX;                      // row length of H in shared memory

// One instance of a resident launch (device memory; written back with the
// outcome).
struct ResInst {
  DGArgs mesh;      // mesh fields (pointers empty)
  double* q;        // state (N), advanced in place
  double* V;        // Krylov basis, (m_max + 1) x ld, FP64: N entries and the tail entry at N
  float* Vh;        // mixed form: FP32 rounding of each basis vector's top part, (m_max + 1) x ld
  double* wv;       // the new Krylov vector (ld)
  double* r;        // dt R(q^n) (N)
  double* acc;      // w(s), the phi-sum so far (N)
  void* z;          // linearisation state (M x stride; FP64, or FP32 in the mixed form)
  float2* qfx;      // mixed form: q^n as float-float pairs (the residual's operand)
  int* flag;        // non-physical state met by the residual (bit 0)
  size_t N, ld;
  size_t onchip;    // shared memory the basis and the vectors need to live on chip (bytes)
  double dt, tol;
  int nsteps, m_max, m_step, iop, max_substeps;
  // outcome
  int status;       // expdg_status of the solve
  int steps_done, krylov_iters, substeps, rejected;
  double err_est;   // largest error estimate of an accepted sub-step
};

// Sum of one value per thread over the CTA, in a fixed order; every thread
// gets the total.  red: NW + 3 doubles of shared memory.  ROOT: thread 0
// also forms sqrt(total) and 1 / sqrt(total) into red[NW + 1], red[NW + 2]
// (one thread: on this GPU an FP64 square root or division issued by every
// thread of the CTA costs a few hundred cycles of the narrow FP64 pipe).
template <int NW, bool ROOT = false>
__device__ double cta_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < NW; ++k) t += red[k];
    red[NW] = t;
    if (ROOT) {
      const double rt = sqrt(t);
      red[NW + 1] = rt;
      red[NW + 2] = 1.0 / rt;
    }
  }
  __syncthreads();
  const double t = red[NW];
  __syncthreads();  // red may be reused at once
  return t;
}

// Sum of x over the warp, the same butterfly on every lane (a fixed order).
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

// 1/k!, k = 0..18 (k! exact in binary64 up to 18!, one rounding each)
constexpr double fact(int k) { return k <= 1 ? 1.0 : k * fact(k - 1); }
__constant__ const double kInvFact[19] = {
    1.0 / fact(0),  1.0 / fact(1),  1.0 / fact(2),  1.0 / fact(3),  1.0 / fact(4),  1.0 / fact(5),  1.0 / fact(6),
    1.0 / fact(7),  1.0 / fact(8),  1.0 / fact(9),  1.0 / fact(10), 1.0 / fact(11), 1.0 / fact(12), 1.0 / fact(13),
    1.0 / fact(14), 1.0 / fact(15), 1.0 / fact(16), 1.0 / fact(17), 1.0 / fact(18)};

// Entry (r, c) of B_j = sum_{i<4, 4j+i<=18} X^i / (4j+i)! (X^0 = I).
__device__ __forceinline__ double pst_block(int j, int r, int c, int k, const double* X, const double* X2,
                                            const double* X3) {
  double b = fma(kInvFact[4 * j + 2], X2[k], fma(kInvFact[4 * j + 1], X[k], (r == c) ? kInvFact[4 * j] : 0.0));
  if (j < 4) b = fma(kInvFact[4 * j + 3], X3[k], b);
  return b;
}

// out = A B (+ B_j when j >= 0), m x m row-major: each entry's sum over l
// split over KS adjacent lanes (shorter dependent chains on the FP64 pipe),
// whole warps in every trip so the shuffles see all lanes.
constexpr int KS = 4;
template <int NT>
__device__ __forceinline__ void mat_mul(const double* A, const double* B, double* out, int m, int j,
                                        const double* X, const double* X2, const double* X3) {
  const int lane = threadIdx.x & 31, total = m * m * KS;
  for (int t0 = threadIdx.x - lane; t0 < total; t0 += NT) {
    const int t = t0 + lane, k = t / KS, part = t - k * KS;
    const bool on = t < total;
    const int r = on ? k / m : 0, c = on ? k - r * m : 0;
    double acc = 0.0;
    if (on)
      for (int l = part; l < m; l += KS) acc = fma(A[r * m + l], B[l * m + c], acc);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (on && part == 0) out[k] = (j >= 0) ? acc + pst_block(j, r, c, k, X, X2, X3) : acc;
  }
}

// y = exp(H_m) e_1 for the m x m leading block of H (row length HC), FP64:
// s = the least s >= 0 with ||H / 2^s||_1 <= 1/2, X = H / 2^s, the degree-18
// Taylor polynomial T(X) by Paterson-Stockmeyer in X^4 (X^2, X^3, X^4, then
// T = B_0 + X^4 (B_1 + X^4 (B_2 + X^4 (B_3 + X^4 B_4))): 7 products for the
// 18 of Horner's rule, the same polynomial), then s squarings.  W: six m x m
// shared buffers.  Every thread of the CTA calls it.
template <int NT>
__device__ void cta_expm_col(const double* H, int m, double* W, double* y) {
  __shared__ double s_norm;
  const int tid = threadIdx.x, mm = m * m;
  double* X = W;
  double* X2 = X + mm;
  double* X3 = X2 + mm;
  double* X4 = X3 + mm;
  double* cur = X4 + mm;
  double* nxt = cur + mm;
  for (int c = tid; c < m; c += NT) {  // column sums of |H|
    double t = 0.0;
    for (int r = 0; r < m; ++r) t += fabs(H[r * HC + c]);
    nxt[c] = t;
  }
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int c = 0; c < m; ++c) mx = fmax(mx, nxt[c]);
    s_norm = mx;
  }
  __syncthreads();
  const double nrm = s_norm;
  const int s = (nrm > 0.5) ? (int)ceil(log2(nrm / 0.5)) : 0;
  const double scale = ldexp(1.0, -s);
  for (int k = tid; k < mm; k += NT) {
    const int r = k / m, c = k - r * m;
    X[k] = H[r * HC + c] * scale;
  }
  __syncthreads();
  mat_mul<NT>(X, X, X2, m, -1, X, X2, X3);
  __syncthreads();
  mat_mul<NT>(X2, X, X3, m, -1, X, X2, X3);
  __syncthreads();
  mat_mul<NT>(X3, X, X4, m, -1, X, X2, X3);
  for (int k = tid; k < mm; k += NT) {  // B_4
    const int r = k / m, c = k - r * m;
    cur[k] = pst_block(4, r, c, k, X, X2, X3);
  }
  __syncthreads();
  for (int jb = 3; jb >= 0; --jb) {
    mat_mul<NT>(X4, cur, nxt, m, jb, X, X2, X3);
    __syncthreads();
    double* sw = cur;
    cur = nxt;
    nxt = sw;
  }
  for (int q = 0; q < s; ++q) {
    mat_mul<NT>(cur, cur, nxt, m, -1, X, X2, X3);
    __syncthreads();
    double* sw = cur;
    cur = nxt;
    nxt = sw;
  }
  for (int r = tid; r < m; r += NT) y[r] = cur[r * m];
  __syncthreads();
}

// float-float split of a double (its top 48 bits), on the integer pipes
__device__ __forceinline__ void split_ff(double x, float& h, float& l) {
  h = f64_to_f32_rn(x);
  l = f64_to_f32_rn(x - f32_to_f64_exact(h));
}

// The resident solve of one instance by one CTA.  MX: the mixed form.
template <int DIM, int P, int EQ, bool MX>
__global__ void __launch_bounds__(dg_threads<DIM, P, 0>()) k_resident(ResInst* list, int n, const Tab tab, size_t onchip_cap) {
  constexpr int NT = dg_threads<DIM, P, 0>(), NW = NT / 32;
  constexpr int EPB = elems_per_block<DIM, P, 0>();
  using TR = typename std::conditional<MX, fx, double>::type;     // residual arithmetic
  using TL = typename std::conditional<MX, float, double>::type;  // linear operator arithmetic
  using SR = DgSmem<DIM, P, EQ, TR, 0>;
  using SL = DgSmem<DIM, P, EQ, TL, 0>;
  if ((int)blockIdx.x >= n) return;
  ResInst& I = list[blockIdx.x];
  const int tid = threadIdx.x;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [H | W (six m x m buffers of exp(H_m); the window pass's partial sums)
  //  | y | red | DG residual smem | DG linear smem | on-chip vectors]
  double* H = reinterpret_cast<double*>(smem_raw);
  double* W = H + (RES_MMAX + 1) * HC;
  double* X = W;  // partial sums of the window pass
  double* y = W + 6 * RES_MMAX * RES_MMAX;
  double* red = y + RES_MMAX + 1;
  unsigned char* dgr = reinterpret_cast<unsigned char*>(red + NW + 3 + 7);
  dgr = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dgr) + 15) & ~uintptr_t(15));
  unsigned char* dgl = dgr + ((SR::bytes() + 15) & ~size_t(15));
  const SR smr(dgr);
  const SL sml(dgl);
  for (int k = tid; k < (P + 1) * (P + 1); k += NT) {
    smr.sD[k] = d_entry<TR>(tab, k);
    sml.sD[k] = d_entry<TL>(tab, k);
  }
  __shared__ int s_flag;
  __shared__ double hs[EXPDG_MAX_IOP + 1];  // window products and ||w||^2 of a classical pass
  static_assert((EXPDG_MAX_IOP + 1) * NT <= 6 * RES_MMAX * RES_MMAX, "partial sums fit W");
  // the operator arguments of the current phase (thread 0 sets them, then a barrier)
  __shared__ DGArgs s_a;
  if (tid == 0) s_a = I.mesh;

  const size_t N = I.N, ld = I.ld, stride = I.mesh.stride;
  const int nelem = I.mesh.nelem, m_max = I.m_max, m_step = I.m_step, iop = I.iop;
  const double dt = I.dt, tol = I.tol, gamma = cst<double>(I.mesh.gamma);
  double* __restrict__ q = I.q;
  double* V = I.V;
  float* Vh = I.Vh;
  double* wv = I.wv;
  double* r = I.r;
  double* acc = I.acc;
  void* zp = I.z;
  if (I.onchip <= onchip_cap) {
    // a small instance: the basis and the vectors in shared memory (a pass
    // over the unknowns then waits on shared-memory latency, not L2's)
    unsigned char* x = dgl + ((SL::bytes() + 15) & ~size_t(15));
    V = reinterpret_cast<double*>(x);
    wv = V + (size_t)(m_max + 1) * ld;
    r = wv + ld;
    acc = r + ld;
    zp = acc + ld;
    Vh = reinterpret_cast<float*>(acc + 2 * ld);
  }
  int iters = 0, subs = 0, rej = 0, status = EXPDG_OK, done = 0;
  double err_max = 0.0;
  __syncthreads();

  for (int step = 0; step < I.nsteps && status == EXPDG_OK; ++step) {
    // linearisation state of q^n (and its float-float copy in the mixed form)
    for (size_t i = tid; i < stride; i += NT)
      linstate_node<DIM, EQ, TL>(q, static_cast<TL*>(zp), stride, gamma, 0, MX ? I.qfx : nullptr, i);
    if (tid == 0) {
      *I.flag = 0;
      s_a.alpha = dt;
      split_ff(dt, s_a.alpha_h, s_a.alpha_l);
      s_a.q = MX ? static_cast<const void*>(I.qfx) : static_cast<const void*>(q);
      s_a.v = nullptr;
      s_a.out = r;
      s_a.status = I.flag;
    }
    __syncthreads();
    // r = dt R(q^n)
    for (int e0 = 0; e0 < nelem; e0 += EPB) {
      dg_group<DIM, P, EQ, TR, false, false, 0, false>(s_a, tab, e0, smr, false);
      __syncthreads();
    }
    if (tid == 0) s_flag = *(volatile int*)I.flag;
    __syncthreads();
    if (s_flag & 1) {
      status = EXPDG_ENONPHYSICAL;
      break;
    }
    double rn2 = 0.0;
    for (size_t i = tid; i < N; i += NT) {
      rn2 = fma(r[i], r[i], rn2);
      acc[i] = 0.0;  // w(0) = c_0 = 0
    }
    cta_sum<NW, true>(rn2, red);
    const double rnorm = red[NW + 1];
    __syncthreads();

    // w = phi_1(dt L) r by sub-steps s -> s + sigma
    double s = 0.0, sigma = 1.0;
    int rej_solve = 0;  // rejected attempts of this Krylov solve
    while (s < 1.0) {
      // eta = 2^-round(log2 ||sigma r||) (sigma a power of two: ||sigma r|| = sigma ||r||)
      const double b1n = sigma * rnorm;
      // eta a power of two: exponent arithmetic, no FP64 pipe work
      const int ex = (b1n == 0.0 || !isfinite(b1n)) ? 0 : (int)rint(log2(b1n));
      const double eta = ldexp(1.0, -ex);
      const double te = ldexp(1.0, ex);  // the start vector's tail entry 1 / eta
      double a2 = 0.0;
      for (size_t i = tid; i < N; i += NT) a2 = fma(acc[i], acc[i], a2);
      if (tid == 0) a2 = fma(te, te, a2);
      cta_sum<NW, true>(a2, red);
      const double beta = red[NW + 1], ib = red[NW + 2];
      __syncthreads();
      for (size_t i = tid; i < N; i += NT) {
        const double v = acc[i] * ib;
        V[i] = v;
        if (MX) Vh[i] = f64_to_f32_rn(v);
      }
      if (tid == 0) V[N] = te * ib;
      for (int k = tid; k < (RES_MMAX + 1) * HC; k += NT) H[k] = 0.0;
      __syncthreads();
      bool ok = false;
      int m = 0;
      double err = 0.0;
      for (int j = 0; j < m_max; ++j) {
        // w = A_hat v_j = [sigma dt L x + eta y_j (sigma r); 0]
        if (tid == 0) {
          s_a.alpha = sigma * dt;
          s_a.alpha_h = f64_to_f32_rn(sigma * dt);
          s_a.alpha_l = 0.0f;
          s_a.q = zp;
          s_a.v = MX ? static_cast<const void*>(Vh + (size_t)j * ld) : static_cast<const void*>(V + (size_t)j * ld);
          s_a.out = wv;
          s_a.status = nullptr;
        }
        __syncthreads();
        for (int e0 = 0; e0 < nelem; e0 += EPB) {
          dg_group<DIM, P, EQ, TL, true, false, 0, MX>(s_a, tab, e0, sml, false);
          __syncthreads();
        }
        ++iters;
        const double* vj = V + (size_t)j * ld;
        const double ey = eta * vj[N] * sigma;
        const int lo = (iop > 0) ? max(0, j - iop + 1) : 0;
        double w0 = 0.0, hprev = 0.0, ihn = 0.0;  // ||w||^2 before, ||w'|| and 1 / ||w'|| after
        if (iop > 0) {
          // window (at most EXPDG_MAX_IOP slots): one classical pass, all the
          // window's products and ||w|| at once, then one update with ||w'||;
          // the window's vectors are orthonormal in exact arithmetic, so this
          // is the modified sweep's projection up to rounding
          const int nw = j - lo + 1;
          double d[EXPDG_MAX_IOP];
#pragma unroll
          for (int c = 0; c < EXPDG_MAX_IOP; ++c) d[c] = 0.0;
          double d0 = 0.0;
          for (size_t k = tid; k <= N; k += NT) {
            double x = (k < N) ? fma(ey, r[k], wv[k]) : 0.0;  // augmentation column; tail: J y = 0
            wv[k] = x;
            d0 = fma(x, x, d0);
#pragma unroll
            for (int c = 0; c < EXPDG_MAX_IOP; ++c)
              if (c < nw) d[c] = fma(V[(size_t)(lo + c) * ld + k], x, d[c]);
          }
          // rows 0..nw-1: the products, row nw: ||w||^2; partial sums in X
          // (free outside the checks), one warp per row, fixed order
#pragma unroll
          for (int c = 0; c < EXPDG_MAX_IOP; ++c)
            if (c < nw) X[c * NT + tid] = d[c];
          X[nw * NT + tid] = d0;
          __syncthreads();
          const int lane = tid & 31;
          for (int row = tid >> 5; row <= nw; row += NW) {
            double t = 0.0;
#pragma unroll
            for (int q2 = 0; q2 < NW; ++q2) t += X[row * NT + q2 * 32 + lane];
            t = warp_sum(t);
            if (lane == 0) hs[row] = t;
          }
          __syncthreads();
          w0 = hs[nw];  // ||w||^2 (the breakdown test compares squares)
          if (tid < nw) H[(lo + tid) * HC + j] = hs[tid];
          double e = 0.0;
          for (size_t k = tid; k <= N; k += NT) {
            double x = wv[k];
            for (int c = 0; c < nw; ++c) x = fma(-hs[c], V[(size_t)(lo + c) * ld + k], x);
            wv[k] = x;
            e = fma(x, x, e);
          }
          cta_sum<NW, true>(e, red);
          hprev = red[NW + 1];
          ihn = red[NW + 2];
          __syncthreads();
        }
        // full orthogonalisation: modified Gram-Schmidt; pass k subtracts
        // h_{k-1} v_{k-1} and forms <v_k, w> (the first pass adds the tail
        // term and forms ||w||)
        for (int i = lo; iop == 0 && i <= j + 1; ++i) {
          const double* vp = (i > lo) ? V + (size_t)(i - 1) * ld : nullptr;
          const double* vi = V + (size_t)i * ld;  // i = j + 1: not read
          double d = 0.0, d0 = 0.0;
          for (size_t k = tid; k <= N; k += NT) {
            double x = wv[k];
            if (i == lo) {
              x = (k < N) ? fma(ey, r[k], x) : 0.0;  // augmentation column; the tail of A_hat v_j is J y = 0
              d0 = fma(x, x, d0);
            } else {
              x = fma(-hprev, vp[k], x);
            }
            wv[k] = x;
            d = fma((i <= j) ? vi[k] : x, x, d);
          }
          if (i == lo) w0 = cta_sum<NW>(d0, red);
          if (i <= j) {
            const double h = cta_sum<NW>(d, red);
            if (tid == 0) H[i * HC + j] = h;
            hprev = h;
          } else {  // ||w|| after the window
            cta_sum<NW, true>(d, red);
            hprev = red[NW + 1];
            ihn = red[NW + 2];
            __syncthreads();
          }
        }
        const double hn = hprev;
        if (tid == 0) H[(j + 1) * HC + j] = hn;
        m = j + 1;
        const bool breakdown = hn * hn <= 1e-26 * w0;  // ||w'|| <= 1e-13 ||w||
        if (!breakdown) {
          const double ih = ihn;
          double* vn = V + (size_t)(j + 1) * ld;
          for (size_t k = tid; k <= N; k += NT) {
            const double v = wv[k] * ih;
            vn[k] = v;
            if (MX && k < N) Vh[(size_t)(j + 1) * ld + k] = f64_to_f32_rn(v);
          }
        }
        __syncthreads();
        if (breakdown || m % m_step == 0 || m == m_max) {
          cta_expm_col<NT>(H, m, W, y);
          err = breakdown ? 0.0 : beta * hn * fabs(y[m - 1]);
          if (breakdown || err <= tol * beta) {
            ok = true;
            break;
          }
        }
      }
      if (!ok) {
        ++rej;
        if (++rej_solve > I.max_substeps) {
          status = EXPDG_EKRYLOV;
          break;
        }
        sigma *= 0.5;
        continue;
      }
      // w(s + sigma) = beta V_m y (top part)
      for (size_t i = tid; i < N; i += NT) {
        double t = 0.0;
        for (int k = 0; k < m; ++k) t = fma(V[(size_t)k * ld + i], y[k], t);
        acc[i] = beta * t;
      }
      __syncthreads();
      s += sigma;
      ++subs;
      err_max = fmax(err_max, err);
      if (m <= m_max / 2) sigma *= 2.0;
      sigma = fmin(sigma, 1.0 - s);
    }
    if (status != EXPDG_OK) break;
    for (size_t i = tid; i < N; i += NT) q[i] += acc[i];
    __syncthreads();
    ++done;
  }
  if (tid == 0) {
    I.status = status;
    I.steps_done = done;
    I.krylov_iters = iters;
    I.substeps = subs;
    I.rejected = rej;
    I.err_est = err_max;
  }
}

template <int DIM, int P, int EQ>
size_t resident_smem() {
  constexpr int NW = dg_threads<DIM, P, 0>() / 32;
  const size_t head = sizeof(double) * ((RES_MMAX + 1) * HC + 6 * RES_MMAX * RES_MMAX + RES_MMAX + 1 + NW + 3 + 7) + 16;
  return head + ((DgSmem<DIM, P, EQ, fx, 0>::bytes() + 15) & ~size_t(15)) + DgSmem<DIM, P, EQ, float, 0>::bytes() + 64;
}
template <int DIM, int P, int EQ>
size_t resident_smem64() {
  constexpr int NW = dg_threads<DIM, P, 0>() / 32;
  const size_t head = sizeof(double) * ((RES_MMAX + 1) * HC + 6 * RES_MMAX * RES_MMAX + RES_MMAX + 1 + NW + 3 + 7) + 16;
  return head + 2 * ((DgSmem<DIM, P, EQ, double, 0>::bytes() + 15) & ~size_t(15)) + 64;
}

// Dynamic shared memory of a class's launch: the fixed part, plus `onchip`
// bytes for the instances whose basis and vectors fit on chip.
template <int DIM, int P, int EQ, bool MX>
size_t resident_base() {
  return MX ? resident_smem<DIM, P, EQ>() : resident_smem64<DIM, P, EQ>();
}

// Largest on-chip vector region a launch of the class can have: the
// per-block opt-in shared memory less the fixed part and 4 KiB for the
// kernel's static shared variables.
template <int DIM, int P, int EQ, bool MX>
size_t resident_onchip_cap() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t base = resident_base<DIM, P, EQ, MX>();
  return ((size_t)optin > base + 4096) ? (size_t)optin - base - 4096 : 0;
}

template <int DIM, int P, int EQ, bool MX>
cudaError_t launch_resident_t(ResInst* list, int n, size_t onchip, const Tab& tab, cudaStream_t s) {
  const size_t base = resident_base<DIM, P, EQ, MX>();
  auto kern = k_resident<DIM, P, EQ, MX>;
  static const cudaError_t configured = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(base + resident_onchip_cap<DIM, P, EQ, MX>()));
  if (configured != cudaSuccess) return configured;
  if (n <= 0) return cudaSuccess;
  if (onchip > resident_onchip_cap<DIM, P, EQ, MX>()) return cudaErrorInvalidValue;
  kern<<<n, dg_threads<DIM, P, 0>(), base + onchip, s>>>(list, n, tab, onchip);
  return cudaGetLastError();
}

// onchip < 0: return the class's on-chip capacity (bytes) instead of launching.
template <int DIM, int EQ, bool MX>
long long launch_resident_p(int p, ResInst* list, int n, long long onchip, const Tab& tab, cudaStream_t s) {
#define EXPDG_RES_CASE(PP)                                                                  \
  case PP:                                                                                  \
    return onchip < 0 ? (long long)resident_onchip_cap<DIM, PP, EQ, MX>()                 \
                      : (long long)launch_resident_t<DIM, PP, EQ, MX>(list, n, (size_t)onchip, tab, s);
  switch (p) {
    EXPDG_RES_CASE(1)
    EXPDG_RES_CASE(2)
    EXPDG_RES_CASE(3)
    EXPDG_RES_CASE(4)
    EXPDG_RES_CASE(5)
    default: return onchip < 0 ? 0 : (long long)cudaErrorInvalidValue;
  }
#undef EXPDG_RES_CASE
}

long long launch_resident(int eq, int dim, int p, bool mx, ResInst* list, int n, long long onchip, const Tab& tab,
                          cudaStream_t s) {
  if (eq == EXPDG_BURGERS && dim == 1)
    return mx ? launch_resident_p<1, EXPDG_BURGERS, true>(p, list, n, onchip, tab, s)
              : launch_resident_p<1, EXPDG_BURGERS, false>(p, list, n, onchip, tab, s);
  if (eq == EXPDG_EULER && dim == 2)
    return mx ? launch_resident_p<2, EXPDG_EULER, true>(p, list, n, onchip, tab, s)
              : launch_resident_p<2, EXPDG_EULER, false>(p, list, n, onchip, tab, s);
  return onchip < 0 ? 0 : (long long)cudaErrorInvalidValue;
}

}  // namespace
}  // namespace expdg

using namespace expdg;

struct expdg_batch {
  struct Class {
    int eq, dim, p;
    bool mx;
    int first, count;  // instances [first, first + count) of the grouped list
    size_t onchip;     // on-chip vector region of the class's launch (bytes; 0: none)
    Tab tab;
  };
  int n = 0;
  std::vector<expdg_config> cfg;
  std::vector<int> pos;          // instance i -> its index in the grouped list
  std::vector<ResInst> h;        // grouped list (host copy)
  ResInst* d = nullptr;          // grouped list (device)
  std::vector<Class> classes;
  std::vector<cudaStream_t> streams;  // one per class
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  std::vector<void*> allocs;
  int device = 0;
  bool ran = false;
};

namespace {

expdg_status batch_check(const expdg_config& c) {
  if (c.scheme != EXPDG_EPI2) return EXPDG_EINVAL;
  if (!((c.eq == EXPDG_BURGERS && c.dim == 1) || (c.eq == EXPDG_EULER && c.dim == 2))) return EXPDG_EINVAL;
  if (c.p < 1 || c.p > 5) return EXPDG_EINVAL;
  if (c.prec != EXPDG_FP64 && c.prec != EXPDG_MIXED) return EXPDG_EINVAL;
  if (c.flux != EXPDG_FLUX_LF) return EXPDG_EINVAL;
  for (int d = 0; d < c.dim; ++d)
    if (c.ne[d] < 1 || !(c.hi[d] > c.lo[d])) return EXPDG_EINVAL;
  if (c.eq == EXPDG_EULER && !(c.gamma > 1.0)) return EXPDG_EINVAL;
  if (!(c.krylov_tol > 0.0) || c.m_max < 1 || c.m_max > EXPDG_BATCH_MAX_KRYLOV || c.m_step < 1) return EXPDG_EINVAL;
  if (c.max_substeps < 0 || c.iop < 0 || c.iop > EXPDG_MAX_IOP) return EXPDG_EINVAL;
  if (!(c.kappa >= 0.0) || !std::isfinite(c.kappa)) return EXPDG_EINVAL;
  if (c.bc != EXPDG_BC_PERIODIC && c.bc != EXPDG_BC_DIRICHLET) return EXPDG_EINVAL;
  if ((c.kappa > 0.0 || c.bc != EXPDG_BC_PERIODIC) && c.eq != EXPDG_BURGERS) return EXPDG_EINVAL;
  return EXPDG_OK;
}

template <typename T>
cudaError_t balloc(expdg_batch* b, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, (n > 0 ? n : 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  b->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaMemset(q, 0, (n > 0 ? n : 1) * sizeof(T));
}

bool device_ptr_of(const void* p, int dev) {
  cudaPointerAttributes at{};
  if (p == nullptr || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}

}  // namespace

extern "C" {

void expdg_batch_destroy(expdg_batch* b) {
  if (!b) return;
  for (cudaStream_t s : b->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (void* p : b->allocs) cudaFree(p);
  delete b;
}

expdg_status expdg_batch_create(const expdg_config* cfgs, int n, expdg_batch** out) {
  if (!out) return EXPDG_EINVAL;
  *out = nullptr;
  if (!cfgs || n < 1) return EXPDG_EINVAL;
  for (int i = 0; i < n; ++i)
    if (batch_check(cfgs[i]) != EXPDG_OK) return EXPDG_EINVAL;
  expdg_batch* b = new expdg_batch();
  b->n = n;
  b->cfg.assign(cfgs, cfgs + n);
  cudaGetDevice(&b->device);
  // group by class, keeping the given order within a class
  std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
  for (int i = 0; i < n; ++i)
    groups[std::make_tuple(cfgs[i].eq, cfgs[i].dim, cfgs[i].p, cfgs[i].prec)].push_back(i);
  b->pos.assign(n, 0);
  b->h.resize(n);
  cudaError_t e = cudaSuccess;
#define BALLOC(call)                                                   \
  do {                                                                 \
    if ((e = (call)) != cudaSuccess) {                                 \
      cudaGetLastError();                                              \
      expdg_batch_destroy(b);                                          \
      return e == cudaErrorMemoryAllocation ? EXPDG_ENOMEM : EXPDG_ECUDA; \
    }                                                                  \
  } while (0)
  int k = 0;
  for (auto& g : groups) {
    expdg_batch::Class c{};
    c.eq = std::get<0>(g.first);
    c.dim = std::get<1>(g.first);
    c.p = std::get<2>(g.first);
    c.mx = std::get<3>(g.first) == EXPDG_MIXED;
    c.first = k;
    c.count = (int)g.second.size();
    double r[MAXP + 1], w[MAXP + 1], D[(MAXP + 1) * (MAXP + 1)];
    build_lgl(c.p, r, w, D);
    fill_tab(c.tab, D, c.p, 1.0 / w[0]);
    for (int i : g.second) {
      const expdg_config& cf = cfgs[i];
      ResInst& I = b->h[k];
      std::memset(&I, 0, sizeof(I));
      b->pos[i] = k++;
      DGArgs& m = I.mesh;
      size_t nelem = 1, np = 1;
      for (int d = 0; d < 3; ++d) {
        const bool used = d < cf.dim;
        m.ne[d] = used ? cf.ne[d] : 1;
        m.two_over_h[d] = make_cst(used ? 2.0 / ((cf.hi[d] - cf.lo[d]) / cf.ne[d]) : 2.0);
        if (used) {
          nelem *= (size_t)cf.ne[d];
          np *= (size_t)(cf.p + 1);
        }
      }
      if (nelem > (size_t)0x7fffffff / np) {
        expdg_batch_destroy(b);
        return EXPDG_EINVAL;
      }
      const int M = (cf.eq == EXPDG_BURGERS) ? 1 : cf.dim + 2;
      m.nelem = (int)nelem;
      m.gamma = make_cst(cf.gamma);
      m.stride = nelem * np;
      m.kappa = make_cst(cf.kappa);
      m.viscous = cf.kappa != 0.0 ? 1 : 0;
      m.dirichlet = (cf.bc == EXPDG_BC_DIRICHLET) ? 1 : 0;
      I.N = (size_t)M * nelem * np;
      I.ld = ((I.N + EXPDG_MAX_PHI + 63) / 64) * 64;
      I.tol = cf.krylov_tol;
      I.m_max = cf.m_max;
      I.m_step = cf.m_step;
      I.iop = cf.iop;
      I.max_substeps = cf.max_substeps;
      const size_t nb = I.ld * (size_t)(cf.m_max + 1);
      BALLOC(balloc(b, &I.V, nb));
      if (c.mx) BALLOC(balloc(b, &I.Vh, nb));
      BALLOC(balloc(b, &I.wv, I.ld));
      BALLOC(balloc(b, &I.r, I.N));
      BALLOC(balloc(b, &I.acc, I.N));
      if (c.mx) {
        float* z = nullptr;
        BALLOC(balloc(b, &z, I.N));
        I.z = z;
        BALLOC(balloc(b, &I.qfx, I.N));
      } else {
        double* z = nullptr;
        BALLOC(balloc(b, &z, I.N));
        I.z = z;
      }
      BALLOC(balloc(b, &I.flag, 1));
      // V ((m_max + 1) ld), wv, r, acc, z (ld each) in FP64, and the FP32
      // shadows of V in the mixed form
      I.onchip = sizeof(double) * ((size_t)(cf.m_max + 1) * I.ld + 4 * I.ld) +
                 (c.mx ? sizeof(float) * (size_t)(cf.m_max + 1) * I.ld : 0) + 64;
    }
    // the class's launch gets the largest region that fits the capacity; the
    // instances that need more keep their vectors in device memory
    const long long cap = launch_resident(c.eq, c.dim, c.p, c.mx, nullptr, 0, -1, c.tab, nullptr);
    c.onchip = 0;
    for (int i : g.second) {
      const size_t need = b->h[b->pos[i]].onchip;
      if ((long long)need <= cap && need > c.onchip) c.onchip = need;
    }
    for (int i : g.second)
      if (b->h[b->pos[i]].onchip > c.onchip) b->h[b->pos[i]].onchip = (size_t)-1;  // stays in device memory
    b->classes.push_back(c);
  }
  BALLOC(balloc(b, &b->d, (size_t)n));
  for (size_t i = 0; i < b->classes.size(); ++i) {
    cudaStream_t s = nullptr;
    BALLOC(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    b->streams.push_back(s);
    cudaEvent_t ev = nullptr;
    BALLOC(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    b->joins.push_back(ev);
  }
  BALLOC(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  BALLOC(cudaDeviceSynchronize());
#undef BALLOC
  *out = b;
  return EXPDG_OK;
}

expdg_status expdg_batch_advance(expdg_batch* b, double* const* q, const double* dt, int nsteps, void* stream) {
  if (!b || !q || !dt || nsteps < 0) return EXPDG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return EXPDG_EINVAL;
  for (int i = 0; i < b->n; ++i)
    if (!device_ptr_of(q[i], dev) || !(dt[i] > 0.0) || !std::isfinite(dt[i])) return EXPDG_EINVAL;
  for (int i = 0; i < b->n; ++i) {
    ResInst& I = b->h[b->pos[i]];
    I.q = q[i];
    I.dt = dt[i];
    I.nsteps = nsteps;
    I.status = EXPDG_OK;
    I.steps_done = I.krylov_iters = I.substeps = I.rejected = 0;
    I.err_est = 0.0;
  }
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(b->d, b->h.data(), sizeof(ResInst) * b->n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaEventRecord(b->fork, s) != cudaSuccess)
    return EXPDG_ECUDA;
  // one launch per class, the classes side by side on their own streams
  for (size_t k = 0; k < b->classes.size(); ++k) {
    const expdg_batch::Class& c = b->classes[k];
    if (cudaStreamWaitEvent(b->streams[k], b->fork, 0) != cudaSuccess) return EXPDG_ECUDA;
    if (launch_resident(c.eq, c.dim, c.p, c.mx, b->d + c.first, c.count, (long long)c.onchip, c.tab,
                        b->streams[k]) != (long long)cudaSuccess) {
      cudaGetLastError();
      return EXPDG_ECUDA;
    }
    if (cudaEventRecord(b->joins[k], b->streams[k]) != cudaSuccess || cudaStreamWaitEvent(s, b->joins[k], 0) != cudaSuccess)
      return EXPDG_ECUDA;
  }
  if (cudaMemcpyAsync(b->h.data(), b->d, sizeof(ResInst) * b->n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return EXPDG_ECUDA;
  b->ran = true;
  for (int i = 0; i < b->n; ++i)
    if (b->h[b->pos[i]].status != EXPDG_OK) return (expdg_status)b->h[b->pos[i]].status;
  return EXPDG_OK;
}

expdg_status expdg_batch_result(const expdg_batch* b, int i, expdg_stats* st, int* steps_done) {
  if (!b || i < 0 || i >= b->n || !b->ran) return EXPDG_EINVAL;
  const ResInst& I = b->h[b->pos[i]];
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->krylov_iters = I.krylov_iters;
    st->substeps = I.substeps;
    st->rejected = I.rejected;
    st->jv_applies = I.krylov_iters;
    st->residual_applies = I.steps_done + (I.status == EXPDG_ENONPHYSICAL ? 1 : 0);
    st->err_est = I.err_est;
  }
  if (steps_done) *steps_done = I.steps_done;
  return (expdg_status)I.status;
}

int expdg_batch_launches(const expdg_batch* b) { return b ? (int)b->classes.size() : 0; }

}  // extern "C"
