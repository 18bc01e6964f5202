// Types shared by the host orchestration and the kernels of the IFNSO library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ifnso {

// Tensor-core tiles: 128 x 256 outputs per tile (one tcgen05 MMA of M = 128,
// N = 256 per 16-wide K step), K blocks of 64 elements (one 128-byte
// swizzled row per operand row).  Square h x h workspace buffers are padded
// to multiples of 256 so that a symmetric 256 x 256 block grid covers them.
constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;
constexpr int HPAD = 256;
constexpr int kSmallH = 128;  // matrices with h <= kSmallH fit the on-chip path (small.cu)

enum EpiKind : int {
  EPI_GRAM = 0,      // T_0 tile -> FP32 buffer (direct + mirrored), sum T_0^2 and tr T_0
  EPI_SQR = 1,       // D_{l+1} = 2 D_l - D_l^2, P -= w_{l+1} D_{l+1}
  EPI_APPLY = 2,     // Y = P A / sqrt(o)
  EPI_NS_GRAM = 3,   // S = X X^T (BF16, direct + mirrored)
  EPI_NS_SQR = 4,    // B = b S + c S^2 (BF16, direct + mirrored)
  EPI_NS_APPLY = 5,  // X <- a X + (B X  or  b S X)
  EPI_GRAM_F8 = 6,   // T_0 from E4M3 copies of A (kind::f8f6f4), rescaled; else as EPI_GRAM
  EPI_SQR_FOLD = 7,  // EPI_SQR with -2 D_l folded into the MMAs (chosen by TcParams::fold_d)
  EPI_APPLY_UPDATE = 8,  // EPI_APPLY whose result updates the weights: W -= lr s Y (TcParams::update)
  EPI_SQR_NORM = 9,      // ||D_1^2||_F^2 into MatScalars::spare[0], nothing stored (Gelfand q = 2)
  EPI_APPLY_F16 = 10,    // EPI_APPLY from FP16 operands: P (one FP16 value) and the scaled FP16 copy A s
  EPI_APPLY_UPDATE_F16 = 11,  // EPI_APPLY_UPDATE from the same FP16 operands
};

// Power-of-two scale s of the FP16 copy A s read by the FP16 product, from
// tr T_0 = ||A||_F^2: max |A_ij| s <= ||A||_F s <= 32768 < 65504 (the largest
// FP16 value), and s within 2^-60..2^60; 1 for a zero or non-finite norm.
__device__ __forceinline__ float f16_copy_scale(double trace) {
  if (!(trace > 0.0) || !(trace < 1e300)) return 1.f;
  int e = static_cast<int>(floor(log2(32768.0 / sqrt(trace))));
  e = e < -60 ? -60 : (e > 60 ? 60 : e);
  return exp2f(static_cast<float>(e));
}

// Per-matrix scalars kept in the workspace (64 bytes).
struct MatScalars {
  double o2;       // sum of squares of T_0 (FP32 partials, FP64 accumulation)
  double trace;    // tr(T_0) = ||A||_F^2
  double s2;       // squared input scale: o = ||T_0||_F (Gram scaling) or ||A||_F^2
  double c0;       // identity weight of the D basis, 1 + sum_l w_l (FP64)
  float inv_s2;    // 1 / s2, rounded once to FP32
  float inv_s;     // 1 / sqrt(s2), rounded once to FP32
  int32_t status;  // IFNSO_DEV_* bits
  uint32_t amax;   // bits of max |A_ij| as a float (E4M3 Gram: its scale); a max of
                   // non-negative floats is a max of their bit patterns
  double spare[2];
};

// Power-of-two scale s with max |A_ij| s in (224, 448]: the E4M3 copy of A
// holds A s (448 is the largest finite E4M3 value).  s is kept within
// 2^-60..2^60 so that 1/s^2 stays a normal FP32 value; 1 for an all-zero A.
__device__ __forceinline__ float e4m3_scale(uint32_t amax_bits) {
  const float amax = __uint_as_float(amax_bits);
  if (!(amax > 0.f) || !(amax < 3.0e38f)) return 1.f;
  int e = static_cast<int>(floorf(log2f(448.f / amax)));
  e = e < -60 ? -60 : (e > 60 ? 60 : e);
  float s = ldexpf(1.f, e);
  if (amax * s > 448.f) s *= 0.5f;  // log2f rounded up across a power of two
  return s;
}
static_assert(sizeof(MatScalars) == 64, "MatScalars layout");

// Coefficients w_1..w_L: either one FP64 vector shared by all matrices or an
// FP32 row per matrix (slot 0 of each row is the identity weight, ignored).
struct CoefTable {
  const double* d64;
  const float* f32;
  int32_t K;
  int32_t stride;
};

__device__ __forceinline__ double coef_at(const CoefTable& t, int m, int l) {
  return t.f32 ? static_cast<double>(t.f32[static_cast<int64_t>(m) * t.stride + l]) : t.d64[l];
}

// Symmetric h_pad x h_pad intermediates (T_0, D_l, P, and S, B of the
// Newton-Schulz baseline) are stored on their 256 x 256 blocks on and above
// the diagonal only: element (i, k) with i / 256 > k / 256 is read as (k, i).
constexpr int kSymA = 1;  // TcProblem::sym: A operand is such a buffer
constexpr int kSymB = 2;  // B operand is such a buffer (then the same one as A)

// One matrix product of a tensor-core pass.  The tensor maps live in global
// memory (64-byte aligned) and are read by TMA directly.
struct TcProblem {
  CUtensorMap mapA[2];  // A-operand sources (rows of the output tile)
  CUtensorMap mapB[2];  // B-operand sources (columns of the output tile)
  CUtensorMap mapT[2];  // the symmetric operand buffers read transposed (boxes 64 x 64)
  int32_t n_kb;         // number of 64-wide K blocks
  int32_t mat;          // matrix index (scalars, coefficients, status)
  int32_t a_mn;         // 1: A operand is MN-major in memory (TMA boxes 64 x 64)
  int32_t b_mn;         // 1: B operand is MN-major in memory
  int32_t out_trans;    // apply: tile element (r, c) is written to out[c][r]
  int32_t rows_out;     // valid extent of out0 in its own layout
  int32_t cols_out;
  int32_t sym;          // kSymA | kSymB
  int64_t ld_out;       // leading dimension of out0/out1 (elements)
  int64_t ld_aux;       // leading dimension of aux0/aux1 and pacc (elements)
  void* out0;
  void* out1;
  const void* aux0;
  const void* aux1;
  float* pacc;
};

static_assert(alignof(TcProblem) % 64 == 0 && sizeof(TcProblem) % alignof(TcProblem) == 0,
              "TcProblem arrays must keep every tensor map 64-byte aligned");

// A pair of 128 x 256 output tiles of one problem: rows [128 tm, 128 tm + 256)
// (tm even; CTA r of the cluster computes tile tm + r), columns
// [256 tn, 256 tn + 256).  flags bit 0: a diagonal 256 x 256 block of a
// symmetric output (stands for itself only; the others also for their
// transpose, which is not stored).
struct WorkItem {
  uint16_t prob;
  uint16_t tm;
  uint16_t tn;
  uint16_t flags;
};

struct MatInfo;

struct TcParams {
  const TcProblem* probs;
  const WorkItem* items;
  int32_t n_items;
  int32_t coef_l;      // EPI_SQR: index l + 1 of the coefficient this pass adds
  int32_t final_pass;  // EPI_SQR: write P (BF16 hi/lo) instead of D_{l+1}
  int32_t ns_step;     // NS epilogues: step index (step 0 applies the input scale)
  int32_t read_lo;     // EPI_SQR: this pass multiplies D_l = hi + lo (split operands)
  int32_t write_lo;    // EPI_SQR: store D_{l+1} as hi + lo (the next pass is split)
  int32_t p_split;     // EPI_SQR final pass / prep: store P as BF16 hi + lo
  int32_t p_mode;      // EPI_SQR: 0 P untouched, 1 P written from c0 I and two terms,
                       // 2 two terms subtracted from P, 3 one term subtracted from P (in L2,
                       // without reading P; the final pass reads it and writes hi + lo),
                       // 4 P written from c0 I, w_1 T_0 / o (read) and two terms
  int32_t feat;        // EPI_SQR: accumulate sum (D_l^2)_ij^2 into MatScalars::spare[0]
  int32_t inject;      // testing aid: CTA 0's producer loads nothing, so its waits run out
  uint32_t wait_ms;    // limit of every pipeline wait (0: the default of ptx.cuh)
  int32_t cta_group;   // 2: MMAs of the CTA pair (M = 256, B halves stay in each CTA);
                       // 1: per-CTA MMAs, each CTA loading the whole B tile
  int32_t fold_d;      // EPI_SQR: the MMAs also add -2 D_l (an identity product), so the
                       // accumulator holds D_l^2 - 2 D_l = -D_{l+1} and the epilogue
                       // does not read D_l (passes whose P update has no D_l term)
  int32_t p_f16;       // EPI_SQR final pass: store P as one FP16 value (for EPI_APPLY_F16)
  int32_t max_stages;  // 0: the whole ring of operand stages; else the stages this pass uses
                       // (fewer operand bytes in flight, for passes whose epilogue loads
                       // or stores compete with them in L2)
  int32_t update;      // EPI_APPLY: out0 holds the weights W (M's shape, also read through
                       // aux0): W <- W - lr sqrt(max(1, rows / cols)) Y instead of Y
  float lr;            // the step size of that update
  // Side work of a squaring pass: part side_part of side_parts equal parts of
  // the FP16 copies M s of side_mats[0 .. side_count) (the copies' 8-value
  // pieces, matrix after matrix) for the FP16 product, written by extra warps
  // of every CTA while the pass runs (side_scal: their scalar records;
  // side_mats nullptr: no side work)
  const MatInfo* side_mats;
  const MatScalars* side_scal;
  int32_t side_count;
  int32_t side_part, side_parts;
  MatScalars* scal;
  CoefTable coef;
  float ns_a, ns_b, ns_c, ns_bcoef;
};

// Per-matrix description used by the SIMT kernels (norms, scalars, prep,
// FP32 products).
struct MatInfo {
  const void* in;
  void* out;
  int64_t rows, cols, ld;  // M's own shape
  int32_t h, w, hpad, trans;
  int32_t on_chip;         // the on-chip path (small.cu) computes this matrix: the tiled passes skip it
  int32_t pad_;
  float* gp;               // h_pad x h_pad FP32: T_0, then P
  void* d[4];              // D buffer 0 hi, lo; D buffer 1 hi, lo
  void* x[2];              // NS: X ping-pong (M's layout, leading dimension xld)
  void* s;                 // NS: S = X X^T
  void* b;                 // NS: B = b S + c S^2
  int64_t xld;
  uint8_t* a8;             // E4M3 Gram: A s (h x w, K-major, leading dimension a8ld bytes)
  int64_t a8ld;
  void* a16;               // FP16 product: M s (M's layout, leading dimension a16ld elements)
  int64_t a16ld;
};

// One matrix of the on-chip path for h <= 128 (small.cu): the whole of
// Algorithm 1 in one CTA.  The tensor maps view the input M itself.
struct SmProblem {
  CUtensorMap mapG;  // the Gram's operand: M K-major (box 64 x 128), or, M tall, M^T MN-major (box 64 x 64)
  CUtensorMap mapY;  // the product's B operand: M MN-major (box 64 x 64), or, M tall, K-major (box 64 x 256)
  void* out;         // Y in M's shape, BF16, leading dimension ld_out
  int64_t ld_out;
  int32_t h, w;      // oriented shape (h <= 128)
  int32_t trans;     // M is tall: A = M^T
  int32_t pad;
};
static_assert(sizeof(SmProblem) % 64 == 0, "SmProblem arrays must keep every tensor map 64-byte aligned");

struct SmParams {
  const SmProblem* probs;
  MatScalars* scal;
  CoefTable coef;
  const int32_t* idx;  // matrix of CTA b: idx[b] (a list of the batch's matrices with h <= 128), or
                       // first + b when idx is null
  int32_t first;    // matrix index of CTA 0 (idx null)
  int32_t L;
  int32_t k_split;  // squarings 1..k_split multiply split (hi + lo) FP16 operands
  int32_t p_split;  // P enters the product as BF16 hi + lo
  int32_t frob;     // scale by ||A||_F^2 instead of ||A A^T||_F
  uint32_t wait_ms;
};

// One matrix of the on-chip Newton-Schulz baseline (h <= 128): views of the
// input A and of two workspace buffers X0, X1 (M's layout) for the Gram
// (mapG) and as the product's B operand and store target (mapY).
struct SmNsProblem {
  CUtensorMap mapG[3];  // A, X0, X1
  CUtensorMap mapY[3];
  void* out;            // Y in M's shape, BF16, leading dimension ld_out
  int64_t ld_out;
  int32_t h, w, trans, pad;
  int32_t pad2[8];
};
static_assert(sizeof(SmNsProblem) % 64 == 0, "SmNsProblem arrays must keep every tensor map 64-byte aligned");

struct SmNsParams {
  const SmNsProblem* probs;
  MatScalars* scal;
  int32_t first;
  int32_t steps;
  int32_t degree;  // 5 quintic, 3 cubic
  uint32_t wait_ms;
  float a, b, c;   // X <- a X + (b S + c S^2) X
};

// ------------------------------------------------------------ launchers
// (defined in tc_gemm.cu / simt.cu / learn.cu; called by api.cu)
// Launches clusters of two CTAs (at most max_clusters, at most one per item;
// items are pairs of tiles, see WorkItem), in the MMA mode p.cta_group.
cudaError_t tc_launch(int epi, int na, int nb, const TcParams& p, int max_clusters, cudaStream_t s);
// Depth of the operand ring of the tensor-core pass with na x nb operand
// sources in MMA mode cg (TcParams::max_stages at or above it changes nothing).
int tc_ring_stages(int na, int nb, int cg);
int tc_smem_bytes(int na, int nb, int cta_group);
// One CTA per matrix first .. first + count - 1 (every one with h <= 128).
cudaError_t launch_small(const SmParams& p, int count, cudaStream_t s);
cudaError_t launch_small_ns(const SmNsParams& p, int count, cudaStream_t s);

cudaError_t launch_norm2(const MatInfo* d_mats, int count, int bf16, double* out,
                         int64_t out_stride, int grid_x, cudaStream_t s);
cudaError_t launch_scalars(const MatInfo* d_mats, int count, MatScalars* scal, CoefTable coef,
                           int L, int scale_frob, int from_norm2, cudaStream_t s);
// d_only: write D_1 only (no P, T_0 kept), for the norm pass of Gelfand scaling.
// write_p (tensor-core path): also write P = c_0 I - w_1 D_1 (FP32) over T_0.
cudaError_t launch_prep(const MatInfo* d_mats, int count, int hpad_max, MatScalars* scal,
                        CoefTable coef, int L, int split, int f32, cudaStream_t s, int d_only = 0,
                        int write_p = 0);
// Gelfand scaling with q = 2: from o = ||T_0||_F and spare[0] = ||(T_0/o)^2||_F^2,
// o <- ||T_0^2||_F^(1/2) = o spare[0]^(1/4), with 1/o and 1/sqrt(o) to match.
cudaError_t launch_gelfand(int count, MatScalars* scal, cudaStream_t s);
// E4M3 Gram: max |A_ij| into MatScalars::amax, then the scaled E4M3 copy of
// A (M or M^T, K-major) into MatInfo::a8.
cudaError_t launch_amax(const MatInfo* d_mats, int count, MatScalars* scal, int grid_x, cudaStream_t s);
// FP16 product: the FP16 copy M s of every input (s = f16_copy_scale(tr T_0)).
cudaError_t launch_cast_f16(const MatInfo* d_mats, int count, const MatScalars* scal, int grid_x, cudaStream_t s);
cudaError_t launch_cast_e4m3(const MatInfo* d_mats, int count, int max_h, int max_w, MatScalars* scal,
                             cudaStream_t s);

struct SgProblem {
  const float* A;  // A operand element (i, k) at A[i * sa0 + k * sa1], zero for i >= a_rows
  const float* B;  // B operand element (j, k) at B[j * sb0 + k * sb1], zero for j >= b_rows
  int64_t sa0, sa1, sb0, sb1;
  int32_t a_rows, b_rows;
  int32_t M, N, K;  // computed output extent M x N, contraction length K
  int32_t mat;
  int32_t out_trans;
  int32_t rows_out, cols_out;
  int64_t ld_out;
  int64_t ld_aux;
  float* out0;
  const float* aux0;
  float* pacc;
};

struct SgParams {
  const SgProblem* probs;
  int32_t coef_l;
  int32_t final_pass;
  int32_t ns_step;
  int32_t pad0;
  MatScalars* scal;
  CoefTable coef;
  float ns_a, ns_b, ns_c, ns_bcoef;
};

cudaError_t sg_launch(int epi, const SgParams& p, int count, int max_m, int max_n, cudaStream_t s);

// Muon momentum of one matrix (rows x cols): M <- beta M + G (FP32, contiguous),
// U <- G + beta M (nesterov) or M, rounded to BF16 (leading dimension ldg, as G).
cudaError_t launch_muon_momentum(const void* g, int64_t ldg, float* m, void* u, int64_t rows, int64_t cols,
                                 float beta, int nesterov, cudaStream_t s);

cudaError_t launch_learn(int L, int iters, int samples, double lr, int step_size, double gamma,
                         uint32_t seed, double cL, double* d_w, cudaStream_t s);
cudaError_t launch_synth_lowrank(void* out, int64_t rows, int64_t cols, int64_t ld, uint32_t seed,
                                 float alpha, float beta, cudaStream_t s);

// coefficient-proposal MLP (mlp.cu)
int mlp_param_count(int K);
cudaError_t mlp_prepare(int n, const float* sigma, const int64_t* offs, const int32_t* hs, const int32_t* ws,
                        float* xs, float* raw, float* stats, int fit, float* z, cudaStream_t s);
cudaError_t mlp_grad(const float* prm, int K, const float* wfix, const float* scale, const float* z,
                     const float* xs, const int64_t* offs, const int32_t* hs, const int32_t* idx, int batch,
                     float* grad_part, float* loss_part, cudaStream_t s);
cudaError_t mlp_reduce_adam(int K, int batch, const float* grad_part, const float* loss_part, float* grad_out,
                            float* loss_out, float* prm, float* m, float* v, int step, float lr, int do_adam,
                            cudaStream_t s);
cudaError_t mlp_batch_idx(int batch, int step, uint32_t seed, int n, int32_t* idx, cudaStream_t s);
cudaError_t mlp_eval(const float* prm, int K, const float* wfix, const float* scale, const float* z, const float* xs,
                     const int64_t* offs, const int32_t* hs, const int32_t* idx, int n, float* e_mlp, float* e_fix,
                     float* coef_out, int32_t* fallback, cudaStream_t s);
cudaError_t mlp_infer(const float* prm, int K, const float* wfix, const float* scale, const float* stats,
                      const MatInfo* mats, MatScalars* scal, int n, float* coef_rows, int row_stride, cudaStream_t s);

void count_launch(int n = 1);

// Set the thread's message returned by ifnso_last_error() (defined in api.cu).
void set_last_error(const char* msg);

}  // namespace ifnso
