// Adjoint of the sampled TR loss w.r.t. every core (FP32).
//
//   L = 1/2 sum_j w_j || X_S(:, j) - G_{n(2)} Z(j, :)^T ||^2,
//   Z(j, :) = vec of P_j = S_1 S_2 ... S_L (slices G_k(i_k) in the cyclic
//   order n+1, ..., n-1; Algorithm 2).
//
// With e = G_{n(2)} Z(j, :)^T - X_S(:, j) and M_j = sum_i w_j e_i G_n(i),
// the product rule on Trace(G_n(i) A_s S_s B_s) gives
//   dL/dG_n(2)(i, :)  += w_j e_i Z(j, :)
//   dL/dS_s           += (B_s M_j A_s)^T,
// A_s = S_1 ... S_{s-1} (prefix), B_s = S_{s+1} ... S_L (suffix).  Each CTA
// handles one sample and recomputes its prefix and suffix products in shared
// memory, so no prefix or suffix product is ever stored.  The per-sample
// terms (the loss, w_j e, Z(j, :) and each slice's R x R term) go to a
// stream-ordered scratch, and three reduction kernels add them in increasing
// j (fixed order, no atomics): the results do not depend on the schedule.
#include "blocks.cuh"
#include "internal.h"

namespace trsgd {

static constexpr int kAdjR = 16;  // max rank
static constexpr int kAdjThreads = 256;

struct AdjArgs {
  int N, n, J;
  int I[kMaxOrder], R[kMaxOrder];
  const int *idx;
  const float *XS;
  const float *w;
  const float *cores[kMaxOrder];
  bool grads;                        // the gradients are wanted
  // per-sample scratch: loss [J], w_j e [J][I_n], Z [J][Q], slice terms [J][L][kAdjR^2]
  float *lossj, *ew, *zj, *cb;
};

__global__ void __launch_bounds__(kAdjThreads) adjoint_kernel(AdjArgs a) {
  __shared__ float S[kMaxOrder][kAdjR * kAdjR];     // slices, column-major R_k x R_{k+1}
  __shared__ float Pre[kMaxOrder][kAdjR * kAdjR];   // prefixes A_s, row-major R_{n+1} x R_k
  __shared__ float Suf[2][kAdjR * kAdjR];           // suffix B_s, row-major R_{k+1} x R_n
  __shared__ float Mm[kAdjR * kAdjR];               // M_j, row-major R_n x R_{n+1}
  __shared__ float T1[kAdjR * kAdjR];               // M A_s, row-major R_n x R_k
  __shared__ float Z[kAdjR * kAdjR];
  __shared__ float red[kAdjThreads / 32];
  extern __shared__ float e_s[];                    // residual, I_n

  const int j = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
  const int N = a.N, n = a.n, L = N - 1;
  const int Rn = a.R[n], Rn1 = a.R[(n + 1) % N], Q = Rn * Rn1, In = a.I[n];
  int order[kMaxOrder];
  for (int s = 0; s < kMaxOrder; ++s) order[s] = (s < L) ? (n + 1 + s) % N : 0;
  const float wj = a.w[j];

  for (int s = 0; s < L; ++s) {
    const int k = order[s], Ra = a.R[k], Rb = a.R[(k + 1) % N];
    const int i = a.idx[(size_t)j * N + k];
    const float *src = a.cores[k] + (size_t)i * Ra * Rb;
    for (int e = tid; e < Ra * Rb; e += NT) S[s][e] = src[e];
  }
  // prefixes: A_0 = I (R_{n+1}), A_{s+1} = A_s S_s
  for (int e = tid; e < Rn1 * Rn1; e += NT) Pre[0][e] = (e / Rn1 == e % Rn1) ? 1.f : 0.f;
  __syncthreads();
  for (int s = 0; s < L; ++s) {
    const int k = order[s], Ra = a.R[k], Rb = a.R[(k + 1) % N];
    if (s + 1 < kMaxOrder) {
      for (int e = tid; e < Rn1 * Rb; e += NT) {
        const int rp = e / Rb, b = e % Rb;
        float acc = 0.f;
        for (int x = 0; x < Ra; ++x) acc = fmaf(Pre[s][rp * Ra + x], S[s][x + b * Ra], acc);
        if (s + 1 < L) Pre[s + 1][rp * Rb + b] = acc;
        else Z[b + rp * Rn] = acc;  // P_j(rp, b): Z(j, b + rp R_n)
      }
    }
    __syncthreads();
  }
  // residual e_i = G_n(i, :) . Z - X_S(i, j), loss
  const float *Gn = a.cores[n];
  float lsum = 0.f;
  for (int i = tid; i < In; i += NT) {
    float acc = 0.f;
    for (int q = 0; q < Q; ++q) acc = fmaf(Gn[(size_t)i * Q + q], Z[q], acc);
    const float e = acc - a.XS[(size_t)j * In + i];
    e_s[i] = e;
    lsum += 0.5f * wj * e * e;
  }
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((tid & 31) == 0) red[tid >> 5] = lsum;
  __syncthreads();
  if (tid == 0) {
    float tot = 0.f;
    for (int x = 0; x < NT / 32; ++x) tot += red[x];
    a.lossj[j] = tot;
  }
  if (!a.grads) return;
  // core n: the terms w e_i Z(q), as w e and Z
  for (int i = tid; i < In; i += NT) a.ew[(size_t)j * In + i] = wj * e_s[i];
  for (int q = tid; q < Q; q += NT) a.zj[(size_t)j * Q + q] = Z[q];
  // M[r][r'] = sum_i w e_i G_n(i)[r][r'] = sum_i w e_i G_n(2)(i, r + r' R_n)
  for (int e = tid; e < Rn * Rn1; e += NT) {
    const int r = e / Rn1, rp = e % Rn1;
    float acc = 0.f;
    for (int i = 0; i < In; ++i) acc = fmaf(e_s[i], Gn[(size_t)i * Q + r + rp * Rn], acc);
    Mm[r * Rn1 + rp] = wj * acc;
  }
  // suffix B_{L-1} = I (R_n)
  int cur = 0;
  for (int e = tid; e < Rn * Rn; e += NT) Suf[0][e] = (e / Rn == e % Rn) ? 1.f : 0.f;
  __syncthreads();
  for (int s = L - 1; s >= 0; --s) {
    const int k = order[s], Ra = a.R[k], Rb = a.R[(k + 1) % N];
    // T1 = M A_s  (R_n x R_k); A_s = Pre[s] (R_{n+1} x R_k)
    for (int e = tid; e < Rn * Ra; e += NT) {
      const int r = e / Ra, x = e % Ra;
      float acc = 0.f;
      for (int y = 0; y < Rn1; ++y) acc = fmaf(Mm[r * Rn1 + y], Pre[s][y * Ra + x], acc);
      T1[r * Ra + x] = acc;
    }
    __syncthreads();
    // this sample's term of slice (x, b): (B_s T1)[b][x], B_s = Suf[cur] (R_{k+1} x R_n)
    float *ck = a.cb + ((size_t)j * L + s) * (kAdjR * kAdjR);
    for (int e = tid; e < Ra * Rb; e += NT) {
      const int x = e % Ra, b = e / Ra;
      float acc = 0.f;
      for (int r = 0; r < Rn; ++r) acc = fmaf(Suf[cur][b * Rn + r], T1[r * Ra + x], acc);
      ck[x + b * Ra] = acc;
    }
    // B_{s-1} = S_s B_s  (R_k x R_n)
    if (s > 0) {
      for (int e = tid; e < Ra * Rn; e += NT) {
        const int x = e / Rn, r = e % Rn;
        float acc = 0.f;
        for (int b = 0; b < Rb; ++b) acc = fmaf(S[s][x + b * Ra], Suf[cur][b * Rn + r], acc);
        Suf[cur ^ 1][x * Rn + r] = acc;
      }
    }
    __syncthreads();
    cur ^= 1;
  }
}

// The loss: each thread sums a contiguous run of samples in order, then
// thread 0 adds the runs in thread order.
__global__ void __launch_bounds__(kAdjThreads) adjoint_loss_kernel(const float *lossj, int J, float *loss) {
  __shared__ float part[kAdjThreads];
  const int tid = threadIdx.x, per = (J + kAdjThreads - 1) / kAdjThreads;
  float acc = 0.f;
  for (int j = tid * per; j < min(J, (tid + 1) * per); ++j) acc += lossj[j];
  part[tid] = acc;
  __syncthreads();
  if (tid == 0) {
    float tot = 0.f;
    for (int x = 0; x < kAdjThreads; ++x) tot += part[x];
    *loss = tot;
  }
}

// dL/dG_n(2)(i, q) = sum_j (w_j e_ij) Z(j, q), j increasing; one thread per entry.
__global__ void adjoint_core_n_kernel(const float *ew, const float *zj, int J, int In, int Q, float *gn) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)In * Q) return;
  const int i = (int)(e / Q), q = (int)(e % Q);
  float acc = 0.f;
  for (int j = 0; j < J; ++j) acc = fmaf(ew[(size_t)j * In + i], zj[(size_t)j * Q + q], acc);
  gn[e] = acc;
}

// dL/dG_k(i) = sum over the samples j with index i on core k of their slice
// terms, j increasing; one thread per slice entry.  s = core k's position in
// the chain.
__global__ void adjoint_slices_kernel(const float *cb, const int *idx, int J, int N, int L, int k, int s, int Ik,
                                      int RR, float *gk) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)Ik * RR) return;
  const int i = (int)(e / RR), el = (int)(e % RR);
  float acc = 0.f;
  for (int j = 0; j < J; ++j)
    if (__ldg(idx + (size_t)j * N + k) == i) acc += cb[((size_t)j * L + s) * (kAdjR * kAdjR) + el];
  gk[e] = acc;
}

cudaError_t launch_sampled_loss_grad(int N, const int *I, const int *R, int n, int J,
                                     const int *idx, const float *XS, const float *w,
                                     const float *const *cores, float *const *grads, float *loss,
                                     cudaStream_t s) {
  if (J <= 0) return cudaSuccess;   // the caller zeroed the loss and the gradients
  AdjArgs a = {};
  a.N = N;
  a.n = n;
  a.J = J;
  for (int k = 0; k < N; ++k) {
    a.I[k] = I[k];
    a.R[k] = R[k];
    a.cores[k] = cores[k];
  }
  a.grads = grads != nullptr;
  a.idx = idx;
  a.XS = XS;
  a.w = w;
  const int L = N - 1, In = I[n], Q = R[n] * R[(n + 1) % N];
  const size_t nl = (size_t)J, new_ = grads ? (size_t)J * In : 0, nz = grads ? (size_t)J * Q : 0,
               nc = grads ? (size_t)J * L * kAdjR * kAdjR : 0;
  float *scratch = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), (nl + new_ + nz + nc) * sizeof(float), s);
  if (e != cudaSuccess) return e;
  a.lossj = scratch;
  a.ew = scratch + nl;
  a.zj = a.ew + new_;
  a.cb = a.zj + nz;
  const size_t dyn = (size_t)In * sizeof(float);
  if (dyn > 48 * 1024) e = cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e == cudaSuccess) {
    adjoint_kernel<<<J, kAdjThreads, dyn, s>>>(a);
    adjoint_loss_kernel<<<1, kAdjThreads, 0, s>>>(a.lossj, J, loss);
    if (grads) {
      const long long nn = (long long)In * Q;
      adjoint_core_n_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(a.ew, a.zj, J, In, Q, grads[n]);
      for (int sp = 0; sp < L; ++sp) {
        const int k = (n + 1 + sp) % N, RR = R[k] * R[(k + 1) % N];
        const long long nk = (long long)I[k] * RR;
        adjoint_slices_kernel<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(a.cb, idx, J, N, L, k, sp, I[k], RR,
                                                                            grads[k]);
      }
    }
    e = cudaGetLastError();
  }
  const cudaError_t f = cudaFreeAsync(scratch, s);
  return e != cudaSuccess ? e : f;
}

}  // namespace trsgd
