// Coefficient learning of Algorithm 1 on the GPU (Sec. 2.3, schedule of
// Sec. 3.1.1), and the Philox4x32-10 generator of the synthetic inputs.
#include <cuda_bf16.h>

#include "common.cuh"

namespace ifnso {

namespace {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (hi0, lo0) = mulhilo(M0, c0), (hi1, lo1) = mulhilo(M1, c2),
// c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), key bumped between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

constexpr uint32_t kTagLearn = 0x4C45524Eu;
constexpr uint32_t kTagLeft = 0x4C524B31u;
constexpr uint32_t kTagRight = 0x4C524B32u;
constexpr uint32_t kTagNoise = 0x4E4F4953u;
constexpr int kMaxL = 30;
constexpr int kLearnThreads = 1024;

// One CTA runs the whole optimisation.  Iteration t: each thread evaluates
// its samples x_j of f(x) = x + sum_{l<L} w_l x t_l + w_L x t_L with
// t_l = (1 - x^2)^(2^(l-1)) (repeated squaring) and w_L = cL - sum_{l<L} w_l
// (Eq. overall_polynomial, cL = e^(1/2)(2^(L/2) - 1)), accumulates the
// gradient 2 (f - 1) (x t_k - x t_L) of sum_j (f(x_j) - 1)^2, the CTA reduces
// it, and threads k < L - 1 take the Adam step of w_k.
__global__ void __launch_bounds__(kLearnThreads, 1)
    k_learn(int L, int iters, int samples, double lr, int step_size, double gamma, uint32_t seed,
            double cL, double* w_out) {
  __shared__ double w[kMaxL], mom[kMaxL], vel[kMaxL];
  __shared__ double red[kLearnThreads / 32][kMaxL];
  const int n = L - 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < kMaxL) {
    w[tid] = 0.0;
    mom[tid] = 0.0;
    vel[tid] = 0.0;
  }
  __syncthreads();
  double p1 = 1.0, p2 = 1.0, lr_t = lr;
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  for (int t = 0; t < iters && n > 0; ++t) {
    if (t > 0 && step_size > 0 && t % step_size == 0) lr_t *= gamma;
    double g[kMaxL];
    for (int k = 0; k < n; ++k) g[k] = 0.0;
    double wl = cL;
    for (int k = 0; k < n; ++k) wl -= w[k];
    for (int j = tid; j < samples; j += blockDim.x) {
      const uint4 r = philox(make_uint4(static_cast<uint32_t>(j), static_cast<uint32_t>(t), 0u, 0u),
                             seed, kTagLearn);
      const double x = (static_cast<double>(r.x >> 5) * 67108864.0 + static_cast<double>(r.y >> 6) + 0.5) *
                       (1.0 / 9007199254740992.0);
      double phi[kMaxL + 1];
      double tl = 1.0 - x * x;
      for (int l = 1; l <= L; ++l) {
        phi[l] = x * tl;
        tl = tl * tl;
      }
      double f = x + wl * phi[L];
      for (int k = 0; k < n; ++k) f += w[k] * phi[k + 1];
      const double e2 = 2.0 * (f - 1.0);
      for (int k = 0; k < n; ++k) g[k] += e2 * (phi[k + 1] - phi[L]);
    }
    for (int k = 0; k < n; ++k) {
      double v = g[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    p1 *= b1;
    p2 *= b2;
    if (tid < n) {
      double gk = 0.0;
      for (int q = 0; q < static_cast<int>(blockDim.x >> 5); ++q) gk += red[q][tid];
      const double m = b1 * mom[tid] + (1.0 - b1) * gk;
      const double v = b2 * vel[tid] + (1.0 - b2) * gk * gk;
      mom[tid] = m;
      vel[tid] = v;
      const double denom = sqrt(v) / sqrt(1.0 - p2) + eps;
      w[tid] = w[tid] - (lr_t / (1.0 - p1)) * m / denom;
    }
    __syncthreads();
  }
  if (tid == 0) {
    double wl = cL;
    for (int k = 0; k < n; ++k) {
      w_out[k] = w[k];
      wl -= w[k];
    }
    w_out[n] = wl;
  }
}

// Rank-32 signal plus noise, one 32-row x 256-column tile per CTA.  The
// factor rows of the tile are generated into shared memory once; element
// (i, j) is fl(fl(fl(alpha * S_ij) + N_ij) * beta) rounded to BF16, with the
// integer S_ij = sum_r L_ir R_jr exact in int32.
__global__ void __launch_bounds__(256) k_synth_lowrank(__nv_bfloat16* out, int64_t rows,
                                                       int64_t cols, int64_t ld, uint32_t seed,
                                                       float alpha, float beta) {
  __shared__ int Ls[32][33];
  __shared__ int Rs[256][33];
  const int64_t i0 = static_cast<int64_t>(blockIdx.y) * 32;
  const int64_t j0 = static_cast<int64_t>(blockIdx.x) * 256;
  auto byte_sum = [](uint32_t v) {
    return static_cast<int>((v & 0xFFu) + ((v >> 8) & 0xFFu) + ((v >> 16) & 0xFFu) + (v >> 24)) - 510;
  };
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int ii = e >> 5, r = e & 31;
    const uint4 u = philox(make_uint4(static_cast<uint32_t>(i0 + ii), static_cast<uint32_t>(r), 0u, 0u),
                           seed, kTagLeft);
    Ls[ii][r] = byte_sum(u.x);
  }
  for (int e = threadIdx.x; e < 256 * 32; e += blockDim.x) {
    const int jj = e >> 5, r = e & 31;
    const uint4 u = philox(make_uint4(static_cast<uint32_t>(j0 + jj), static_cast<uint32_t>(r), 0u, 0u),
                           seed, kTagRight);
    Rs[jj][r] = byte_sum(u.x);
  }
  __syncthreads();
  const int jj = threadIdx.x;
  const int64_t j = j0 + jj;
  if (j >= cols) return;
  for (int ii = 0; ii < 32; ++ii) {
    const int64_t i = i0 + ii;
    if (i >= rows) break;
    int s = 0;
#pragma unroll
    for (int r = 0; r < 32; ++r) s += Ls[ii][r] * Rs[jj][r];
    const uint4 u = philox(make_uint4(static_cast<uint32_t>(j), static_cast<uint32_t>(i), 0u, 0u), seed,
                           kTagNoise);
    const int nz = static_cast<int>((u.x & 0xFFFFu) + (u.x >> 16) + (u.y & 0xFFFFu) + (u.y >> 16)) - 131070;
    float t = __fmul_rn(alpha, static_cast<float>(s));
    t = __fadd_rn(t, static_cast<float>(nz));
    t = __fmul_rn(t, beta);
    out[i * ld + j] = __float2bfloat16_rn(t);
  }
}

}  // namespace

cudaError_t launch_learn(int L, int iters, int samples, double lr, int step_size, double gamma,
                         uint32_t seed, double cL, double* d_w, cudaStream_t s) {
  k_learn<<<1, kLearnThreads, 0, s>>>(L, iters, samples, lr, step_size, gamma, seed, cL, d_w);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_synth_lowrank(void* out, int64_t rows, int64_t cols, int64_t ld, uint32_t seed,
                                 float alpha, float beta, cudaStream_t s) {
  dim3 grid(static_cast<unsigned>((cols + 255) / 256), static_cast<unsigned>((rows + 31) / 32));
  k_synth_lowrank<<<grid, 256, 0, s>>>(static_cast<__nv_bfloat16*>(out), rows, cols, ld, seed, alpha,
                                       beta);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ifnso
