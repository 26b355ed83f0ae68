// Internal declarations shared by the libfctn translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "fctn.h"

// Digits of a contraction plan's output index.  A chain intermediate of m of
// the N factors keeps its m modes and the m (N - m) bonds to the rest, at most
// m (N - m + 1) labels: 20 at N = 8 (m = 4 or 5), so 24 covers every order.
#define FCTN_MAXD 24
#define FCTN_MAXC 8   // digits of its contracted index
#define FCTN_CON_TABLE 4096  // contracted-index offsets kept in shared memory

// Programmatic dependent launch.  A kernel launched by launch_pdl may
// become resident while its predecessor in the stream is still running: it
// first lets its own successor launch, then waits for the predecessor's
// completion (and memory) before it touches any data, so stream order is
// kept while the launch latency overlaps the predecessor's tail.
__device__ __forceinline__ void pdl_prologue() {
#if defined(__CUDA_ARCH__)
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
#endif
}
// Whether launch_pdl sets the programmatic attribute (per host thread): on
// only around chains that no concurrent branch needs SMs for, since a kernel
// resident early holds its SM resources while it waits.
extern thread_local bool g_pdl;
struct PdlScope {
  bool prev;
  explicit PdlScope(bool on) : prev(g_pdl) { g_pdl = on; }
  ~PdlScope() { g_pdl = prev; }
};
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = g_pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Sum over z = 0 .. n - 1 of part[z * MN + e] in split order with Neumaier's
// compensation (about twice the FP32 precision; FP64 adds run at 1/64 of the
// FP32 rate), eight loads in flight: the fixed-order reduce of K-split partials.
__device__ __forceinline__ float split_sum(const float* __restrict__ part, int n, int64_t MN, int64_t e) {
  float s = 0.f, c = 0.f;
  int z = 0;
  auto add = [&](float v) {
    const float t = s + v;
    c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
    s = t;
  };
  for (; z + 8 <= n; z += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = part[(int64_t)(z + u) * MN + e];
#pragma unroll
    for (int u = 0; u < 8; ++u) add(v[u]);
  }
  for (; z < n; ++z) add(part[(int64_t)z * MN + e]);
  return s + c;
}

// Index plan of one tensor contraction (Definition 3): the output is dense
// row-major over `out_ext`; each output digit walks operand A with `a_str`
// and operand B with `b_str` (0 = not present); the contracted digits walk
// A with `ca_str` and B with `cb_str`.  B == nullptr turns the kernel into a
// permute (generalized transposition, Definition 1).
struct ContractPlan {
  int nout, ncon;
  int64_t out_ext[FCTN_MAXD];
  int64_t a_str[FCTN_MAXD], b_str[FCTN_MAXD];
  int64_t con_ext[FCTN_MAXC];
  int64_t ca_str[FCTN_MAXC], cb_str[FCTN_MAXC];
  int64_t out_size, con_size;
};

// View of X_(k) as (pre, I_k, post): element (i, j) with j = a*post + b sits at
// a*I_k*post + i*post + b.
struct ModeView {
  int64_t pre, I, post;
};

// Split-K contraction D = M [M ; X_(k)]^T (Gram block then RHS block); the
// Gram block is left out (gcols = 0) when the Gram comes from the operand
// Grams of the pair form (FactGram).
struct GramPlan {
  int64_t s, I, Pk;     // M: s x Pk row-major; X_(k): I x Pk through `xv`
  ModeView xv;
  int64_t gcols;        // Gram columns of D: s, or 0
  int64_t ncols;        // gcols + I
  int tiles_r, tiles_c; // 64 x 64 output tiles
  int ksplit;           // number of K chunks
  int64_t kchunk;       // columns of M per chunk (multiple of 32)
};

// Pair form of a merged tensor (see kernels_fused.cu):
//   M[sigma, j] = sum_kappa L[loff(j) + lo[sigma] + lk[kappa]] * R[roff(j) + ro[sigma] + rk[kappa]]
// j is decoded row-major over `ext` (the modes t != k, ascending); each digit
// adds `lstr` (`rstr`) elements to loff (roff).  tab = {lo[s], ro[s], lk[K], rk[K]}.
struct PairPlan {
  int nd;
  int64_t ext[FCTN_MAX_ORDER];
  int64_t lstr[FCTN_MAX_ORDER], rstr[FCTN_MAX_ORDER];
  int Ljs, Rjs;  // row lengths of L and R (elements staged per column)
  int K;         // contracted length
  const int* tab;
};

// Gram of M_k from the Grams of its pair operands.  With rows sigma of M_k
// split as (L offset, R offset) = (a(sigma), b(sigma)) and F_L[(a, kappa), jL]
// = L[loffL(jL) + offL[a K + kappa]] (jL over the modes held by L; F_R alike):
//   G[sigma, sigma'] = sum_{kappa, kappa'} HL[a K + kappa, a' K + kappa'] HR[b K + kappa, b' K + kappa'],
//   HL = F_L F_L^T, HR = F_R F_R^T.
struct FactGram {
  int use;
  int nL, nR, K, rl, rr;  // rl = nL K rows of F_L, rr = nR K rows of F_R
  int JL, JR;             // columns of F_L, F_R
  const int* tab;         // {offL[rl], offR[rr], a[s], b[s], colL[JL], colR[JR]}: F_L[r][j] = L[colL[j] + offL[r]]
};
void launch_fact_gram_f32(const FactGram& f, const float* L, const float* R, float* HL, float* HR, int s, double* Gd,
                          float* Gs, cudaStream_t st);
void launch_fact_gram_f64(const FactGram& f, const double* L, const double* R, double* HL, double* HR, int s,
                          double* Gd, cudaStream_t st);

// ---- kernels_tc.cu ------------------------------------------------------------
// Column groups of the tensor-core Gram kernel: each CTA computes, for all
// 128-row blocks of M_k, the Gram columns [0, mw) (if mw > 0) and the
// right-hand-side columns of X rows [xi0, xi0 + xw), within 512 TMEM columns.
#define TC_MAX_GROUPS 8
struct TcGroup {
  int mw, xi0, xw, width;
};
struct TcPlan {
  int n_mb, n_groups, BK, tmem_cols;
  uint32_t a_bytes, x_bytes;
  size_t smem;
  TcGroup groups[TC_MAX_GROUPS];
};
int tc_plan(const PairPlan& p, const GramPlan& g, int precision, TcPlan* tp);
void launch_gram_tc(const PairPlan& p, const float* L, const float* R, const float* X, float* part,
                    const GramPlan& g, const TcPlan& tp, int precision, float* Mout, int* status, cudaStream_t st);

// ---- kernels_fused.cu -------------------------------------------------------
void launch_gram_fused_f32(const PairPlan& p, const float* L, const float* R, const float* X, float* part,
                           const GramPlan& g, float* Mout, cudaStream_t st);
void launch_gram_fused_f64(const PairPlan& p, const double* L, const double* R, const double* X, double* part,
                           const GramPlan& g, double* Mout, cudaStream_t st);
void launch_xupdate_fused_f32(const PairPlan& p, const float* L, const float* R, const float* Ak, float* X,
                              const uint32_t* bits, double rho, const GramPlan& g, double* red, cudaStream_t st);
void launch_xupdate_fused_f64(const PairPlan& p, const double* L, const double* R, const double* Ak, double* X,
                              const uint32_t* bits, double rho, const GramPlan& g, double* red, cudaStream_t st);
size_t gram_fused_smem(const PairPlan& p, int s, int bk, int elem);
int gram_fused_bk(const PairPlan& p, int s, int elem);
size_t xupdate_fused_smem(const PairPlan& p, int s, int cb, int elem);
int xupdate_fused_cb(const PairPlan& p, int s, int elem);

// ---- fctn_api.cu -------------------------------------------------------------
// Record `msg` as the calling thread's last error (fctn_last_error) and return code.
int fctn_internal_fail(int code, const char* msg);
// Serving hooks: queue one sweep and an asynchronous copy of the stop-test
// values {rel, objective, data term, nonfinite flag, status, t} into
// `pinned` (host, 6 doubles); the handle's stream.
int fctn_internal_sweep_async(fctn_handle* h, double* pinned);
cudaStream_t fctn_internal_stream(fctn_handle* h);
// Grouped sweeps (serving): one sweep's kernels and stop-test copy issued
// eagerly on the handle's stream (for a stream capture that joins it), or
// only the sweep's host bookkeeping (when a captured group graph that already
// holds this sweep is launched again); the key of the next sweep's kernel
// sequence (equal keys: the same kernels with the same arguments).
int fctn_internal_sweep_eager(fctn_handle* h, double* pinned);
int fctn_internal_sweep_dry(fctn_handle* h, double* pinned);
uint64_t fctn_internal_sweep_key(fctn_handle* h);
// After a sweep whose stop-test change was rel_change: a TF32 / BF16 handle
// with finish_fp32_at > 0 turns to the FP32 products once rel_change <= it.
void fctn_internal_after_sweep(fctn_handle* h, double rel_change);

// ---- kernels_sgemm.cu -------------------------------------------------------
// Table-driven FP32 contraction C[cm[m] + cn[n]] = sum_k A[am[m] + ak[k]] B[bn[n] + bk[k]]
// (offsets in elements, all < 2^31); a K split writes dense partials
// (ksplit x M x N) that are summed in split order.
struct SgShape {
  int M, N, K, ksplit, kchunk;
  int a_mfast, b_nfast;  // loader lanes run along m (n) when that digit is contiguous in A (B), else along k
  int round_tf32;        // C rounded to the nearest TF32 value (a tensor-core operand)
};
struct SgTabs {
  const int *am, *cm, *bn, *cn, *ak, *bk;
};
void sg_shape(int M, int N, int K, SgShape* sh, int split_ctas = 0);  // split_ctas: CTA target of a K split
size_t sg_part_elems(const SgShape& sh);
void launch_sgemm(const SgShape& sh, const SgTabs& t, const float* A, const float* B, float* C, float* part,
                  cudaStream_t st);
// C = sum over the K split (in split order) of the partials [z][M][N] of a split contraction.
void launch_sg_reduce(const SgShape& sh, const SgTabs& t, const float* part, float* C, cudaStream_t st);
// The same contraction on the tensor cores (TF32, operands gathered through
// the tables and rounded to nearest TF32): launch shape, partial elements,
// launches (2 with a K split), launch (A, B, tables as for launch_sgemm).
struct TccShape {
  SgShape sh;            // M, N, K, loader directions, rounding of C; K split of this kernel
  int BN, S;             // columns per CTA (multiple of 16, <= 128), pipeline stages
  int round_a, round_b;  // operands A, B (as launch_tcc takes them) the kernel rounds to TF32
                         // (0: already rounded by their producer)
  int flip;              // sh describes the transposed product C^T = B A^T (the launch swaps the roles)
};
void tcc_shape(const SgShape& sg, int split_ctas, TccShape* ts);
size_t tcc_part_elems(const TccShape& ts);
int tcc_launches(const TccShape& ts);
void launch_tcc(const TccShape& ts, const SgTabs& t, const float* A, const float* B, float* C, float* part,
                int* status, cudaStream_t st);
// Yd = Yraw + rho A_old, Ys = float(Yd) (n = I s); Gd = double(Gs) after symmetrising Gs.
void launch_finish_rhs(const float* Yraw, const double* Aold, double rho, double* Yd, float* Ys, int64_t n,
                       cudaStream_t st);
void launch_finish_gram(float* Gs, double* Gd, int s, cudaStream_t st);
// Transposed / padded copies (dst leading dimension ldd), optionally rounded
// to TF32 or converted to BF16: operands of the tensor-core GEMMs.
void launch_transpose_f32(const float* src, int64_t rows, int64_t cols, int64_t lds, float* dst, int64_t ldd,
                          int round_tf32, cudaStream_t st);
void launch_copy_f32(const float* src, int64_t rows, int64_t cols, int64_t lds, float* dst, int64_t ldd,
                     int round_tf32, cudaStream_t st);
void launch_transpose_bf16(const float* src, int64_t rows, int64_t cols, int64_t lds, __nv_bfloat16* dst,
                           int64_t ldd, cudaStream_t st);
void launch_copy_bf16(const float* src, int64_t rows, int64_t cols, int64_t lds, __nv_bfloat16* dst, int64_t ldd,
                      cudaStream_t st);

// ---- kernels_chol.cu --------------------------------------------------------
// Shifted-Cholesky solve of Eq. 5 (FCTN_SOLVE_CHOL): floor(I / 2) + 1 groups
// of basis rows sharing lam mu_i + rho; per group the packed factor of
// G + c I and the inverses of its 32 x 32 diagonal blocks.
int chol_groups(int I);
bool chol_supported(int s);
size_t chol_factor_floats(int I, int s);
size_t chol_dinv_floats(int I, int s);
// L, Dinv of every group from the FP32 Gram G (s x s); c0, c1: the stencil of L_k.
void launch_chol_factor(const float* G, int I, int s, double lam, double c0, double c1, double rho, float* L,
                        float* Dinv, int* status, cudaStream_t st);
// Rows of W (I x s) with W_i (G + c_i I) = Rt_i (Rt = Q^T R), from the factors of launch_chol_factor.
void launch_chol_subst(const float* Rt, int I, int s, const float* L, const float* Dinv, float* W, int* status,
                       cudaStream_t st);
// Products with the L_k basis (FP32, I x I times I x s): mode 0 out32 = Qm B;
// 1: A64 = Qm B; 2: A64 += Qm B (modes 1, 2 also write Ac = float(A64) and
// Alo = float(A64 - Ac)).
void launch_basis_gemm(int mode, const float* Qm, const float* B, int I, int s, float* out32, double* A64, float* Ac,
                       float* Alo, cudaStream_t st);
// H = A^T A (s x s) for A (I x s) row-major FP32.
void launch_gram_at(const float* A, int I, int s, float* H, cudaStream_t st);
// FP32 R = Yd - lam L A - rho A - A G with A = Ac + Alo, the A G products summed in double-float arithmetic.
void launch_resid_df(const double* Yd, const double* A64, const float* Ac, const float* Alo, const float* G, int I,
                     int s, double lam, double rho, double c0, double c1, float* R, cudaStream_t st);

// ---- kernels_tma.cu ---------------------------------------------------------
// D[M x N] = A[M x K] B[N x K]^T on tcgen05 with TMA-fed operands (both
// K-major); see kernels_tma.cu.  Epilogue modes:
enum { TG_PARTIAL = 0,   // out[z][row][col] (dense M x N per K split z)
       TG_STORE = 1,     // out[row * ldo + col]
       TG_XUPDATE = 2 }; // rows j, columns i of F^T = (A_(1) M_1)^T: Eq. 10 on X_(1)[i, j]
struct TgArgs {
  int M, N, K;     // extents; K beyond the operands' tensor maps reads zeros
  int BN, S;       // columns per CTA (multiple of 16, <= 256), pipeline stages
  int kchunk;      // K per split (multiple of the 128-byte chunk)
  int ksplit;
  int mode;
  float* out;
  int64_t ldo;
  // TG_XUPDATE: X (I_1 x P_1, row-major), observation bits, rho; transposed
  // copy XT (P_1 x ldt, rounded to TF32 when round_tf32) and, for the BF16
  // precision, BF16 copies Xb (I_1 x P_1) and XTb (P_1 x ldt); FP64 partial
  // sums per CTA {||dX||^2, ||X_old||^2, ||X_new - F||^2} into red
  float* X;
  const uint32_t* bits;
  int64_t P0;
  double rho;
  float* XT;
  int64_t ldt;
  __nv_bfloat16* Xb;
  __nv_bfloat16* XTb;
  int round_tf32;  // TG_XUPDATE: XT rounded to TF32; TG_STORE: out rounded to TF32
  double* red;
  int* status;
};
// Tensor map of a row-major operand (rows x cols, leading dimension ld
// elements, 16-byte multiple) for the GEMM: boxes of 128 bytes of K by
// box_rows rows, 128-byte swizzle.  elem: 4 (FP32 / TF32) or 2 (BF16).
int tg_make_map(void* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int elem, int box_rows);
// Unswizzled FP32 map (box box_rows x box_cols, zero fill outside the matrix).
int tma_map_f32(void* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_cols, int box_rows);
size_t tg_smem_bytes(int BN, int S);
// Launch; bf16 selects the BF16 operands and MMA kind.
void launch_tg_gemm(const void* mapA, const void* mapB, const TgArgs& a, int bf16, cudaStream_t st);
void tg_shape(int M, int N, int K, int elem, int want_ctas, TgArgs* a);  // BN, S, kchunk, ksplit
// out[e] = sum over the K split of part[z * MN + e] (split order, FP64), e < MN.
void launch_tg_reduce(const float* part, int ksplit, int64_t MN, float* out, cudaStream_t st);

// ---- kernels_quality.cu ----------------------------------------------------
// PSNR and SSIM (Sec. 4) of X against the truth Y, both (rows x ncol)
// row-major with rows = I_1 I_2 (slice index = column); out = {psnr, ssim}.
size_t quality_work_doubles(int64_t ncol, int nblocks);
void launch_quality_f32(const float* X, const float* Y, int64_t rows, int64_t ncol, double c1, double c2,
                        double* work, int nblocks, double* out, cudaStream_t st);
void launch_quality_f64(const double* X, const double* Y, int64_t rows, int64_t ncol, double c1, double c2,
                        double* work, int nblocks, double* out, cudaStream_t st);

// ---- kernels_contract.cu ---------------------------------------------------
void launch_contract_f32(const float* A, const float* B, float* out, const ContractPlan& p, cudaStream_t s);
void launch_contract_f64(const double* A, const double* B, double* out, const ContractPlan& p, cudaStream_t s);
void launch_laplacian_basis(int64_t I, double delta, int sign, double* Q, float* Qf, double* QT, float* QTf, double* Lam,
                            cudaStream_t s);
void launch_init_x_mask_f32(const float* Y, const uint8_t* mask, float* X, uint32_t* bits, int64_t n, cudaStream_t s);
void launch_init_x_mask_f64(const double* Y, const uint8_t* mask, double* X, uint32_t* bits, int64_t n, cudaStream_t s);
void launch_convert_f64_to_f32(const double* in, float* out, int64_t n, cudaStream_t s);
void launch_convert_f32_to_f64(const float* in, double* out, int64_t n, cudaStream_t s);

// ---- kernels_gram.cu -------------------------------------------------------
// Sum the ksplit partials in a fixed order; write G (s x s), Y = Yraw + rho*A_old
// (I x s) in double and, if Gs/Ys are non-null, single-precision copies.
void launch_reduce_gram_rhs_f32(const float* partials, const GramPlan& g, const double* A_old, double rho,
                                double* Gd, double* Yd, float* Gs, float* Ys, cudaStream_t s);
void launch_reduce_gram_rhs_f64(const double* partials, const GramPlan& g, const double* A_old, double rho,
                                double* Gd, double* Yd, cudaStream_t s);
// X update of Eq. 10 fused with F = A_(k) M (reuse path): writes X in place and
// per-block FP64 partial sums {||dX||^2, ||X_old||^2, ||X_new - F||^2}.
int xupdate_blocks(const GramPlan& g);
void launch_xupdate_f32(const float* Ak, const float* M, float* X, const uint32_t* bits, double rho,
                        const GramPlan& g, double* red, cudaStream_t s);
void launch_xupdate_f64(const double* Ak, const double* M, double* X, const uint32_t* bits, double rho,
                        const GramPlan& g, double* red, cudaStream_t s);

// ---- kernels_solve.cu ------------------------------------------------------
// Symmetric eigendecomposition of the Gram by one-sided Jacobi (one CTA).
// C (s x s, column j = eigenvector j) is read as the warm start when warm != 0
// and overwritten with the result; Phi gets the eigenvalues.  work: 3 s^2.
// *status: FCTN_E_SINGULAR if min Phi + tmin <= 0; *used: sweeps taken
// (minus the sweeps taken if the sweep limit ran out, which is not an error).
// With `rec` (eig_record_floats(s) floats) and 128 < s <= 224 the FP32 route
// is the large block-ordered Jacobi (eig_launches kernels, work 4 s^2).
void launch_eig_f32(const float* G, float* C, float* Phi, float* work, int s, int warm, int max_sweeps,
                    double tmin, int* status, int* used, cudaStream_t st, float* rec = nullptr, double tol = 0.0);
size_t eig_record_floats(int s);
int eig_launches(int s, int warm, int recorded);
// The two stages of the cluster eigensolver for FP32 Grams with 64 < s <= 256
// (eig_is_big), for callers that time them apart: the warm-start products
// (eig_big_prep_launches kernels; work: 4 s^2 floats) and the Jacobi sweeps on
// one cluster of 8 CTAs (kernels_eigc.cu), which write Phi and C.
bool eig_is_big(int s);
void launch_eig_big_prep(const float* G, const float* C, float* work, int s, cudaStream_t st);
int eig_big_prep_launches();
void launch_eig_big_jacobi(const float* G, float* C, float* Phi, float* work, int s, int warm, int max_sweeps,
                           double tmin, double tol, int* status, int* used, cudaStream_t st);
// ---- kernels_eigc.cu: B (s x s) and, warm, V (s x s, column j = eigenvector
// guess j; null = identity) -> Phi, C; *used as in launch_eig_f32.
size_t eigc_smem_bytes(int s);
void launch_eigc(const float* Bin, const float* Vin, float* Phi, float* C, int s, int max_sweeps, double tmin,
                 double tol, int* status, int* used, cudaStream_t st);
void launch_eig_f64(const double* G, double* C, double* Phi, double* work, int s, int warm, int max_sweeps,
                    double tmin, int* status, int* used, cudaStream_t st);
// Eq. 8 by row blocks.  fwd: W = (((Q^T R) C) / T) C^T.  bwd: A = Q W into
// A64 (= or +=) and Ac; with Rout != null (accumulate = 0 only) also the
// FP64 residual of Eq. 5, Rout = Yd - lam L A - rho A - A Gd, for the new A.
void launch_solve_fwd_f32(const float* QT, const float* R, const float* C, const double* LamL, const float* Phi,
                          double lam, double rho, int I, int s, float* W, int* status, cudaStream_t st);
void launch_solve_fwd_f64(const double* QT, const double* R, const double* C, const double* LamL, const double* Phi,
                          double lam, double rho, int I, int s, double* W, int* status, cudaStream_t st);
void launch_solve_bwd_f32(const float* Q, const float* W, int I, int s, int accumulate, double* A64, float* Ac,
                          const double* Yd, const double* Gd, double lam, double rho, double c0, double c1, float* Rout,
                          int* status, cudaStream_t st);
void launch_solve_bwd_f64(const double* Q, const double* W, int I, int s, int accumulate, double* A64, double* Ac,
                          const double* Yd, const double* Gd, double lam, double rho, double c0, double c1,
                          double* Rout, int* status, cudaStream_t st);
// FP64 residual of Eq. 5: R = Y - lam L A - rho A - A G (one CTA per row)
void launch_resid_f32(const double* Y, const double* A, const double* G, int I, int s, double lam, double rho,
                      double c0, double c1, float* R, cudaStream_t st);
void launch_resid_f64(const double* Y, const double* A, const double* G, int I, int s, double lam, double rho,
                      double c0, double c1, double* R, cudaStream_t st);
// asymmetric extrapolation A <- A + alpha (A - beta A_old) of the FP64 master and its compute copy
void launch_extrap_f32(double* A, const double* Aold, double alpha, double beta, float* Ac, int64_t n,
                       cudaStream_t st);
void launch_extrap_f64(double* A, const double* Aold, double alpha, double beta, double* Ac, int64_t n,
                       cudaStream_t st);
// trace term lam/2 tr(A^T L A) for one factor (A: I x s double) -> out[0]
// Trace terms lambda_k / 2 tr(A_(k)^T L_k A_(k)) of every factor (Eq. 2), one launch.
struct TraceArgs {
  const double* A[FCTN_MAX_ORDER];
  int64_t I[FCTN_MAX_ORDER], s[FCTN_MAX_ORDER];
  double c0[FCTN_MAX_ORDER], c1[FCTN_MAX_ORDER], lam[FCTN_MAX_ORDER];
};
void launch_trace_all(const TraceArgs& a, int N, double* out, cudaStream_t st);
// finalize: stats[0]=rel, [1]=objective, [2]=data term, [3]=nonfinite flag
void launch_finalize(const double* red, int nblocks, const double* traces, int N, double* stats, cudaStream_t st);
