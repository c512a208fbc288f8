// Internal declarations shared by the libexpdg translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/expdg.h"

namespace expdg {

// Programmatic dependent launch: a kernel launched with pdl_launch may start
// while the previous kernel in its stream is finishing; it must execute
// griddep_wait() before touching any memory that kernel reads or writes.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Signal that this block's share of the work is done, so the dependent grid may
// be scheduled (it still waits in griddep_wait for this grid's completion).
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = grid;
  lc.blockDim = block;
  lc.dynamicSmemBytes = smem;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, kern, static_cast<KArgs>(args)...);
}

constexpr int MAXP = EXPDG_MAX_ORDER;
constexpr int MMAX = EXPDG_MAX_KRYLOV;
constexpr int RED_THREADS = 256;
constexpr int DOT_CHUNK = 8;          // basis vectors per block row in the multi-dot kernel

// Reference-element data handed to the DG kernels by value (kernel parameter
// space is constant memory; the kernels copy D into shared memory).
// A constant of the operator in the kernels' compute types: FP64 (d) and its
// float-float split (h, the FP32 value, plus l).  Each kernel reads the form
// of its own type, so no thread converts an FP64 constant on the narrow FP64
// pipe (a conversion costs as much there as an FP64 multiply).
struct Cst {
  double d;
  float h, l;
};
inline Cst make_cst(double x) {
  const float h = (float)x;
  return Cst{x, h, (float)(x - (double)h)};
}

// Tile classes of the DG operator kernels: CTAs of about 256 (0, the
// default), 128 (1) or 512 (2) threads, one thread per node.
__host__ __device__ constexpr int tile_threads(int tk) { return tk == 1 ? 128 : (tk == 2 ? 512 : 256); }
inline int tile_elems_per_block(int np, int tk) { return tile_threads(tk) / np > 0 ? tile_threads(tk) / np : 1; }

struct Tab {
  double D[(MAXP + 1) * (MAXP + 1)];   // row-major l_j'(r_i) for the context's order
  float Dh[(MAXP + 1) * (MAXP + 1)];   // its float-float split
  float Dl[(MAXP + 1) * (MAXP + 1)];
  Cst lift;                            // 1 / w_0
};

// D (row-major, (p+1)^2 entries) and 1 / w_0 into a Tab, with their splits.
inline void fill_tab(Tab& t, const double* D, int p, double lift) {
  for (int k = 0; k < (p + 1) * (p + 1); ++k) {
    const Cst c = make_cst(D[k]);
    t.D[k] = c.d;
    t.Dh[k] = c.h;
    t.Dl[k] = c.l;
  }
  t.lift = make_cst(lift);
}

// Arguments of one DG operator apply (see DgForm below for the types of
// q, v and the outputs).
//   residual: out = alpha * R(q)
//   linear:   out = alpha * L(q) v  +  aug
//   aug (Krylov augmented matrix, only when paug > 0):
//     out      += eta * sum_{k=1}^{paug} tail[k-1] * W[paug+1-k]
//     out_tail  = J tail   (upper shift; written by block 0)
// Scalars of the operator applies of one Krylov sub-step, kept in device
// memory (KState) so the launches of an Arnoldi segment do not change between
// sub-steps (they are replayed as CUDA graphs).
struct JvScalars {
  double alpha;  // sigma tau
  double eta;    // tail scale of the augmented matrix
  float alpha_h; // alpha as float-float
  float alpha_l;
  float eta_f;   // eta in FP32 (a power of two: exact)
};

struct DGArgs {
  const void* q;         // T*: residual state q, or linearisation state z of qt
  const void* v;         // T*: linear input vector (top part)
  double alpha;
  float alpha_h;         // alpha as float-float (mixed form)
  float alpha_l;
  double* out;           // FP64 form output
  float* out_h;          // mixed form output (float-float)
  float* out_l;
  int paug;
  double eta;
  float eta_f;           // eta in FP32 (a power of two: exact)
  const double* tail_d;  // tail of the input basis vector (paug entries) or nullptr
  const float* tail_h;
  const float* tail_l;
  const double* W_d[EXPDG_MAX_PHI + 1];  // W[i] = b_i, i = 1..paug
  const float* W_h[EXPDG_MAX_PHI + 1];
  const float* W_l[EXPDG_MAX_PHI + 1];
  const float* W_f[EXPDG_MAX_PHI + 1];   // FP32 copies of b_i (FP64 storage with FP32 arithmetic)
  double* out_tail_d;
  float* out_tail_h;
  float* out_tail_l;
  int* status;           // bit 0: non-physical state met (residual)
  int ne[3];
  int nelem;
  Cst two_over_h[3];
  Cst gamma;
  size_t stride;         // unknowns per field = nelem * Np
  Cst kappa;             // viscosity (1D Burgers; 0: inviscid)
  int viscous;           // kappa != 0
  int dirichlet;         // zero Dirichlet data at both ends (1D Burgers)
  const double* src;     // residual: forcing added to R (FP64, N values) or nullptr
  int roe;               // Euler: Roe flux (the linearisation state then ends with sqrt(rho))
  const JvScalars* scal; // linear: alpha and eta read from here instead of the fields above (or nullptr)
  // Linear: the linearisation state was written by a launch that completed
  // before this launch's predecessor started (inside an Arnoldi step), so it
  // is read before griddepcontrol.wait.  0: read after the wait.
  int z_early;
  int tile;              // tile class of the mixed-form operator apply: CTAs of about 256 (0), 128 (1), 512 (2) threads
};

// A vector in the FP64 form (d) or the float-float form (h + l).
struct Vec {
  double* d;
  float* h;
  float* l;
};

// Krylov basis: vector i at d + i*ld (FP64 and mixed forms) or h/l + i*ld
// (float-float form).  Mixed form: h + i*ld is the FP32 shadow plane of
// vector i (its rounding, read by the FP32 operator apply; the operator's FP32
// output lands there too).
struct Basis {
  double* d;
  float* h;
  float* l;
  size_t ld;
  __host__ __device__ Vec at(int i) const {
    Vec v;
    v.d = d ? d + (size_t)i * ld : nullptr;
    v.h = h ? h + (size_t)i * ld : nullptr;
    v.l = l ? l + (size_t)i * ld : nullptr;
    return v;
  }
};

// Device-resident scalars of one Krylov solve.  H(i, j) = H[j * (MMAX + 1) + i].
// The fields from `red` to the end are read back by the host as one block.
struct KState {
  double H[(MMAX + 1) * MMAX];
  double qcoef[MMAX + 1];   // s_k: delayed re-orthogonalisation coefficients of u_j
  double ucoef[MMAX + 1];   // z_k - (c/r) s_k: projection coefficients of the next vector
  double ycoef[MMAX + 1];   // beta * y_i for the final combination
  double yprev[MMAX + 1];   // y = exp(H_m) e_1 of the previous check (mixed-form rule)
  JvScalars jv;             // alpha and eta of the current sub-step (written by the start kernel)
  double vscale[MMAX + 1];  // basis vector i = vscale_i * slot i (incomplete orthogonalisation; 1 otherwise)
  float2 vsf[MMAX + 1];     // vscale as float-float (h, l): the float-float update reads these
  double wnp[2];            // ||w_j|| by the parity of j (incomplete orthogonalisation, breakdown scale)
  int mprev;                // m of the previous check (0: none)
  int pad2;
  double cu;                // c / r (coefficient of u_j in the next vector)
  double inv_r;             // 1 / ||u_j re-orthogonalised||
  double wnorm;             // ||A_hat q_j|| estimate (happy-breakdown scale)
  unsigned int counter;     // last-block ticket of the reduction kernels
  unsigned int pad0;
  // ---- host-visible block ----
  double red[8];            // results of the norms kernel
  double beta;              // ||[c_0; e_P / eta]|| of the sub-step (computed on the device when adaptive)
  double eta;               // tail scale of the sub-step (likewise)
  double err;               // error estimate at the last check
  double norm1;             // 1-norm of the last H_m
  int accept;               // set by the phi kernel
  int m_eff;                // Krylov dimension used by the last phi kernel
  int breakdown_at;         // first m with a happy breakdown (0: none)
  int squarings;            // scaling exponent used by the last phi kernel
  int status;               // bit 0: non-physical state met by a residual
  int pad1;
};

// ---- DG operators (dg_1d.cu, dg_2d.cu, dg_3d.cu) ----
// Arithmetic and storage of one operator apply.
enum DgForm {
  DG_F64 = 0,     // FP64 in, FP64 arithmetic, FP64 out (the FP64 form, and every form's
                  // residual but the float-float form's)
  DG_F32_FF = 1,  // linear operator: FP32 input vector, FP32 arithmetic, float-float
                  // output (the float-float form)
  DG_F32_MX = 2   // linear operator: FP32 input vector, FP32 arithmetic, output in FP32
                  // (a.out_h) or widened exactly to FP64 (a.out); FP64 augmentation
                  // tail (the mixed form)
};
// form: a DgForm.  Returns the launch error.
cudaError_t launch_dg_1d(bool linear, int form, int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s);
cudaError_t launch_dg_2d(bool linear, int form, int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s);
cudaError_t launch_dg_3d(bool linear, int form, int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s);
// The Roe-flux kernels (Euler; dg_roe_1d.cu, dg_roe_2d.cu, dg_roe_3d.cu), reached
// through launch_dg_Nd when a.roe is set.
cudaError_t launch_dg_roe_1d(bool linear, int form, int p, const DGArgs& a, const Tab& t, cudaStream_t s);
cudaError_t launch_dg_roe_2d(bool linear, int form, int p, const DGArgs& a, const Tab& t, cudaStream_t s);
cudaError_t launch_dg_roe_3d(bool linear, int form, int p, const DGArgs& a, const Tab& t, cudaStream_t s);
// Residual in float-float (a.q: interleaved float-float state, out_h / out_l):
// the mixed form's R, FP64-grade on the FP32 pipes.
cudaError_t launch_dg_fx_1d(int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s);
cudaError_t launch_dg_fx_2d(int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s);
cudaError_t launch_dg_fx_3d(int eq, int p, const DGArgs& a, const Tab& t, cudaStream_t s);
cudaError_t launch_dg_roe_fx_1d(int p, const DGArgs& a, const Tab& t, cudaStream_t s);
cudaError_t launch_dg_roe_fx_2d(int p, const DGArgs& a, const Tab& t, cudaStream_t s);
cudaError_t launch_dg_roe_fx_3d(int p, const DGArgs& a, const Tab& t, cudaStream_t s);
// Euler: z = (u, H, a), or (u, H, sqrt(rho)) with roe.
cudaError_t launch_linstate_1d(int eq, bool fp32, const double* q, void* z, size_t stride, double gamma, int roe,
                               float* qfx, cudaStream_t s);
cudaError_t launch_linstate_2d(int eq, bool fp32, const double* q, void* z, size_t stride, double gamma, int roe,
                               float* qfx, cudaStream_t s);
cudaError_t launch_linstate_3d(int eq, bool fp32, const double* q, void* z, size_t stride, double gamma, int roe,
                               float* qfx, cudaStream_t s);

// ---- Krylov and vector kernels (krylov.cu); ff selects the float-float form ----
// Storage form of the incomplete-orthogonalisation kernels: FP64 basis, float-float
// basis, or FP64 basis with FP32 shadow planes and the operator output in FP32.
enum KForm { KF_F64 = 0, KF_FF = 1, KF_MX = 2 };
// partial-sum buffer entries needed by the reduction kernels
size_t reduction_scratch_entries();
// out = sum_k a[k] x[k] (k < nx <= 5; x[k] with null pointers counts as 0), n entries
cudaError_t launch_lincomb(bool use_ff, Vec out, int nx, const Vec* x, const double* a, size_t n, cudaStream_t s);
// ks->red[k] = ||x_k||^2 (k < nx <= 5; null x[k] gives 0), n entries each
// dev_P >= 0: also eta = 2^-round(log2 max_{1<=i<=P} ||x_i||) and
// beta = sqrt(||x_0||^2 + (P > 0 ? 1/eta^2 : 0)) into KState (no host read needed).
cudaError_t launch_norms(bool use_ff, KState* ks, void* part, int nx, const Vec* x, size_t n, int dev_P,
                         cudaStream_t s);
// 2^-round(log2 nrm) (1 for nrm <= 0 or not finite), the same on host and device.
__host__ __device__ inline double tail_scale_of(double nrm) {
  if (!(nrm > 0.0) || !(nrm < 1.0 / 0.0)) return 1.0;
  int e = 0;
  const double f = frexp(nrm, &e);  // nrm = f 2^e, f in [1/2, 1)
  return ldexp(1.0, -(f >= 0.70710678118654752440 ? e : e - 1));
}
// format conversions (these use the FP64 pipe; only at API and step boundaries)
cudaError_t launch_to_f32(float* out, const double* x, size_t n, cudaStream_t s);
cudaError_t launch_f64_to_ff(Vec out, const double* x, size_t n, cudaStream_t s);
cudaError_t launch_ff_to_f64(double* out, Vec x, size_t n, cudaStream_t s);
// FP64 -> interleaved float-float pairs (out[2i], out[2i+1] = high, low part)
cudaError_t launch_f64_to_fx(float* out, const double* x, size_t n, cudaStream_t s);
// Arnoldi start: u_0 = [b0; e_P / eta] (b0 null: zero top; an FP64 basis with an FP32
// shadow plane (U.h) gets u_0's rounding there too); clears the Krylov scalars;
// vscale_0 = s0 (1 / beta for incomplete orthogonalisation, else 1), vscale_i = 1 for i > 0.
// mode 0: eta and s0 as given; 1: eta from KState, s0 = 1 / beta (0 when beta = 0:
// the zero start vector of incomplete orthogonalisation); 2: eta from KState, s0 = 1.
cudaError_t launch_start(bool use_ff, KState* ks, Basis U, Vec b0, size_t N, int P, double eta, double s0,
                         double alpha, int mode, cudaStream_t s);
// Arnoldi step j by classical Gram-Schmidt with delayed re-orthogonalisation
// (DCGS2).  On entry basis slots 0..j-1 hold the orthonormal q_i, slot j the
// once-orthogonalised u_j, slot j+1 the operator image w = A_hat u_j.
//   dots:   s = Q^T u_j, z = Q^T w, alpha = |u_j|^2, gamma = u_j.w, delta = |w|^2;
//           r = sqrt(alpha - |s|^2); H(:, j-1) += s, H(j, j-1) = r;
//           H(k, j) = (z_k - sum_i s_i H(k, i)) / r, H(j, j) = (c - s_{j-1} r) / r,
//           c = (gamma - s.z) / r.
//   update: q_j = (u_j - Q s) / r -> slot j;
//           u_{j+1} = (w - Q z - c q_j) / r -> slot j+1 (and its FP32 rounding to the
//           shadow plane of an FP64 basis that has one); H(j+1, j) = |u_{j+1}|
//           (provisional until the next step's correction); happy breakdown
//           when |u_{j+1}| <= 1e-13 |A_hat q_j| (recorded in breakdown_at).
cudaError_t launch_dots(bool use_ff, KState* ks, void* part, Basis U, int j, size_t n_aug, cudaStream_t s);
cudaError_t launch_update(bool use_ff, KState* ks, void* part, Basis U, int j, size_t n_aug, cudaStream_t s);
// Arnoldi step j by incomplete orthogonalisation over the window of the last
// iop basis vectors, i = lo..j, lo = max(0, j - iop + 1) (1 <= iop <= EXPDG_MAX_IOP).
// Slot i holds an unnormalised vector, v_i = c_i slot_i with c_i = vscale_i =
// 1 / ||slot_i||; on entry slot j+1 holds w' = A_hat slot_j (= A_hat v_j / c_j).
//   iom_dots:   per-block partial sums of <slot_i, w'> (window) and |w'|^2.
//   iom_update: every block sums those and ||slot_j||^2 (the previous update's
//               partials): c_j, H(j, j-1) = ||slot_j||, H(i, j) = c_i c_j <slot_i, w'>;
//               slot j+1 = c_j w' - sum_i H(i, j) v_i (in place), per-block partials of
//               its norm; happy breakdown when ||slot_j|| <= 1e-13 ||w_{j-1}||.
// kf (KForm): KF_MX reads the top N entries of w' in FP32 from the shadow plane
// of slot j+1 (its P tail entries in FP64) and writes slot j+1 in FP64 and its
// FP32 rounding to the shadow plane.
cudaError_t launch_iom_dots(int kf, int iop, KState* ks, void* part, Basis U, int j, size_t N, size_t n_aug,
                            cudaStream_t s);
cudaError_t launch_iom_update(int kf, int iop, KState* ks, void* part, Basis U, int j, size_t N, size_t n_aug,
                              cudaStream_t s);
// Blocks of an incomplete-orthogonalisation update launch (0 for an invalid iop).
int iom_update_blocks(int kf, int iop, size_t n_aug);
// FP64 phi kernel: E = exp(H_m) (Taylor-18 scaling and squaring), y = E e_1, error estimate,
// acceptance (forced when force_accept), ycoef_i = beta y_i vscale_i.  Acceptance: Saad's
// estimate beta h_{m+1,m} |y_m| <= tol beta; with diff_rule also when the change
// from the previous check, beta |y - [y_prev; 0]|, is <= tol beta.
// iom_part: the reduction scratch when the basis comes from incomplete
// orthogonalisation (h_{m,m-1} is then finished from the last update launch's
// partials; iom_gu = that launch's blocks, iom_kf its KForm), else nullptr.
// ff_arith: float-float arithmetic on the FP32 pipes (the mixed form), else FP64.
// pair: also exp(H_{m-1}) e_1 in the same launch (m >= 2; on a cluster of two
// groups of CTAs, one matrix each, where such clusters fit the GPU, else both
// packed on one group for m <= 49), so that the change with diff_rule is the
// one since m - 1; otherwise since the previous check (y_prev, m_prev).
cudaError_t launch_phi(KState* ks, int m, double beta, double tol, int force_accept, int diff_rule,
                       const void* iom_part, int iom_kf, int iom_gu, bool ff_arith, bool pair, cudaStream_t s);
// out = base + sum_{i < m_eff} ycoef_i u_i (first N entries; base may be null).
// out and base may each be FP64 (d) or float-float (h, l).
// if_accepted: write nothing unless the last phi kernel accepted.
cudaError_t launch_combine(bool use_ff, const KState* ks, Basis U, Vec base, Vec out, size_t N, bool if_accepted,
                           cudaStream_t s);

}  // namespace expdg
