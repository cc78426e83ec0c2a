// Learned disentangler initialiser (an extra beside the paper's identity start,
// Sec. 6): an FP32 MLP 16 -> 128 -> 128 -> 16 with tanh, mapping a two-site
// reduced density matrix (row-major 4 x 4) to an antisymmetric generator
// A = (M - M^T)/2 and u = expm(A) in SO(4).
//
// Kernels (CUDA cores, FP32): dense layers with tanh, the matrix exponential
// of each 4 x 4 generator by scaling and squaring with a degree-12 Taylor
// polynomial (Moler and Van Loan, "Nineteen dubious ways...", method 3), the
// loss mean ||u - u_target||_F^2, its gradient through expm by the Frechet
// derivative L(A^T, G) read off the exponential of the 8 x 8 block matrix
// [[A^T, G], [0, A^T]] (Van Loan 1978; Higham 2008, Thm 3.6 / eq. 10.15),
// weight gradients reduced over the batch in a fixed order, and Adam
// (Kingma and Ba 2015) with bias correction.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mlp.h"

namespace attn {

namespace {

constexpr int NI = 16, NH = 128, NO = 16;

// y[b][o] = act(sum_i W[o][i] x[b][i] + bias[o])
__global__ void dense_kernel(const float* W, const float* bias, const float* x, float* y, int B, int nin, int nout,
                             int act_tanh) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * nout) return;
  const int b = idx / nout, o = idx % nout;
  float s = bias[o];
  for (int i = 0; i < nin; ++i) s = fmaf(W[o * nin + i], x[b * nin + i], s);
  y[idx] = act_tanh ? tanhf(s) : s;
}

// exp of an n x n matrix (row-major, in place) by scaling and squaring + Taylor
template <int n>
__device__ void expm_ss(float* A) {
  float norm = 0.f;  // 1-norm
  for (int j = 0; j < n; ++j) {
    float c = 0.f;
    for (int i = 0; i < n; ++i) c += fabsf(A[i * n + j]);
    norm = fmaxf(norm, c);
  }
  int s = 0;
  while (norm > 0.5f && s < 30) {
    norm *= 0.5f;
    ++s;
  }
  const float sc = ldexpf(1.f, -s);
  float X[n * n], T[n * n], R[n * n], tmp[n * n];
  for (int i = 0; i < n * n; ++i) {
    X[i] = A[i] * sc;
    T[i] = (i / n == i % n) ? 1.f : 0.f;
    R[i] = T[i];
  }
  for (int k = 1; k <= 12; ++k) {  // T <- T X / k ; R += T
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        float acc = 0.f;
        for (int q = 0; q < n; ++q) acc = fmaf(T[i * n + q], X[q * n + j], acc);
        tmp[i * n + j] = acc / (float)k;
      }
    for (int i = 0; i < n * n; ++i) {
      T[i] = tmp[i];
      R[i] += T[i];
    }
  }
  for (int t = 0; t < s; ++t) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        float acc = 0.f;
        for (int q = 0; q < n; ++q) acc = fmaf(R[i * n + q], R[q * n + j], acc);
        tmp[i * n + j] = acc;
      }
    for (int i = 0; i < n * n; ++i) R[i] = tmp[i];
  }
  for (int i = 0; i < n * n; ++i) A[i] = R[i];
}

// per sample: A = (M - M^T)/2, u = expm(A); optional loss and dL/dM
__global__ void head_kernel(const float* Mout, int B, float* u_out, const double* ut, float* loss_part, float* gM) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* M = Mout + b * 16;
  float A[16], U[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) A[i * 4 + j] = 0.5f * (M[i * 4 + j] - M[j * 4 + i]);
  for (int i = 0; i < 16; ++i) U[i] = A[i];
  expm_ss<4>(U);
  for (int i = 0; i < 16; ++i) u_out[b * 16 + i] = U[i];
  if (!ut) return;
  float G[16], l = 0.f;
  for (int i = 0; i < 16; ++i) {
    const float d = U[i] - (float)ut[b * 16 + i];
    l += d * d;
    G[i] = 2.f * d / (float)B;
  }
  loss_part[b] = l / (float)B;
  // Frechet derivative L(A^T, G) = upper-right block of expm([[A^T, G], [0, A^T]])
  float Z[64];
  for (int i = 0; i < 64; ++i) Z[i] = 0.f;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      Z[i * 8 + j] = A[j * 4 + i];
      Z[(i + 4) * 8 + (j + 4)] = A[j * 4 + i];
      Z[i * 8 + (j + 4)] = G[i * 4 + j];
    }
  expm_ss<8>(Z);
  float GA[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) GA[i * 4 + j] = Z[i * 8 + (j + 4)];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) gM[b * 16 + i * 4 + j] = 0.5f * (GA[i * 4 + j] - GA[j * 4 + i]);
}

// gx[b][i] = (sum_o g[b][o] W[o][i]) * (1 - h[b][i]^2) when h given (tanh layer below)
__global__ void back_input_kernel(const float* W, const float* g, const float* h, float* gx, int B, int nin, int nout) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * nin) return;
  const int b = idx / nin, i = idx % nin;
  float s = 0.f;
  for (int o = 0; o < nout; ++o) s = fmaf(g[b * nout + o], W[o * nin + i], s);
  gx[idx] = h ? s * (1.f - h[idx] * h[idx]) : s;
}

// gW[o][i] = sum_b g[b][o] x[b][i]; gb[o] = sum_b g[b][o]  (fixed order over b)
__global__ void back_weight_kernel(const float* g, const float* x, float* gW, float* gb, int B, int nin, int nout) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nout * nin) {
    const int o = idx / nin, i = idx % nin;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s = fmaf(g[b * nout + o], x[b * nin + i], s);
    gW[idx] = s;
  }
  if (idx < nout) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += g[b * nout + idx];
    gb[idx] = s;
  }
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  m[i] = b1 * m[i] + (1.f - b1) * gi;
  v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
  const float mh = m[i] / c1, vh = v[i] / c2;
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void to_f32_kernel(const double* s, float* d, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = (float)s[i];
}

__global__ void sum_kernel(const float* a, int n, float* out) {
  if (threadIdx.x || blockIdx.x) return;
  float s = 0.f;
  for (int i = 0; i < n; ++i) s += a[i];
  *out = s;
}

inline int g1(int n) { return (n + 255) / 256; }  // blocks of 256 threads
inline int g128(int n) { return (n + 127) / 128; }  // blocks of 128 threads

}  // namespace

// parameter layout: W1[128][16] b1[128] W2[128][128] b2[128] W3[16][128] b3[16]
static const size_t OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
                    OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH, NPARAM = OFF_B3 + NO;

size_t mlp_param_count() { return NPARAM; }

void Mlp::ensure(int B) {
  if (B <= cap) return;
  x.reserve(sizeof(float) * B * NI);
  h1.reserve(sizeof(float) * B * NH);
  h2.reserve(sizeof(float) * B * NH);
  mo.reserve(sizeof(float) * B * NO);
  u.reserve(sizeof(float) * B * 16);
  gm.reserve(sizeof(float) * B * NO);
  g2.reserve(sizeof(float) * B * NH);
  g1b.reserve(sizeof(float) * B * NH);
  lp.reserve(sizeof(float) * (B + 1));
  ut.reserve(sizeof(double) * B * 16);
  xin.reserve(sizeof(double) * B * 16);
  cap = B;
}

void Mlp::forward(int B) {
  const float* P = params.as<float>();
  cudaStream_t s = ctx->stream;
  dense_kernel<<<g1(B * NH), 256, 0, s>>>(P + OFF_W1, P + OFF_B1, x.as<float>(), h1.as<float>(), B, NI, NH, 1);
  dense_kernel<<<g1(B * NH), 256, 0, s>>>(P + OFF_W2, P + OFF_B2, h1.as<float>(), h2.as<float>(), B, NH, NH, 1);
  dense_kernel<<<g1(B * NO), 256, 0, s>>>(P + OFF_W3, P + OFF_B3, h2.as<float>(), mo.as<float>(), B, NH, NO, 0);
  ctx->launches += 3;
}

void Mlp::upload_inputs(int B, const double* rho_host, const double* ut_host) {
  ensure(B);
  cudaStream_t s = ctx->stream;
  ATTN_CHECK_CUDA(cudaMemcpyAsync(xin.p, rho_host, sizeof(double) * B * 16, cudaMemcpyHostToDevice, s));
  to_f32_kernel<<<g1(B * 16), 256, 0, s>>>(xin.as<double>(), x.as<float>(), B * 16);
  ctx->launches++;
  if (ut_host) ATTN_CHECK_CUDA(cudaMemcpyAsync(ut.p, ut_host, sizeof(double) * B * 16, cudaMemcpyHostToDevice, s));
}

void Mlp::predict(int B, const double* rho_host, double* u_host) {
  upload_inputs(B, rho_host, nullptr);
  forward(B);
  head_kernel<<<g128(B), 128, 0, ctx->stream>>>(mo.as<float>(), B, u.as<float>(), nullptr, nullptr, nullptr);
  ctx->launches++;
  std::vector<float> hu((size_t)B * 16);
  ATTN_CHECK_CUDA(cudaMemcpyAsync(hu.data(), u.p, sizeof(float) * hu.size(), cudaMemcpyDeviceToHost, ctx->stream));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  for (size_t i = 0; i < hu.size(); ++i) u_host[i] = hu[i];
}

// loss and parameter gradient (into grad) for the uploaded batch
float Mlp::loss_grad(int B) {
  const float* P = params.as<float>();
  float* G = grad.as<float>();
  cudaStream_t s = ctx->stream;
  forward(B);
  head_kernel<<<g128(B), 128, 0, s>>>(mo.as<float>(), B, u.as<float>(), ut.as<double>(), lp.as<float>(), gm.as<float>());
  sum_kernel<<<1, 1, 0, s>>>(lp.as<float>(), B, lp.as<float>() + B);
  // layer 3
  back_weight_kernel<<<g1(NO * NH), 256, 0, s>>>(gm.as<float>(), h2.as<float>(), G + OFF_W3, G + OFF_B3, B, NH, NO);
  back_input_kernel<<<g1(B * NH), 256, 0, s>>>(P + OFF_W3, gm.as<float>(), h2.as<float>(), g2.as<float>(), B, NH, NO);
  // layer 2
  back_weight_kernel<<<g1(NH * NH), 256, 0, s>>>(g2.as<float>(), h1.as<float>(), G + OFF_W2, G + OFF_B2, B, NH, NH);
  back_input_kernel<<<g1(B * NH), 256, 0, s>>>(P + OFF_W2, g2.as<float>(), h1.as<float>(), g1b.as<float>(), B, NH, NH);
  // layer 1
  back_weight_kernel<<<g1(NH * NI), 256, 0, s>>>(g1b.as<float>(), x.as<float>(), G + OFF_W1, G + OFF_B1, B, NI, NH);
  ctx->launches += 7;
  float l = 0.f;
  ATTN_CHECK_CUDA(cudaMemcpyAsync(&l, lp.as<float>() + B, sizeof(float), cudaMemcpyDeviceToHost, s));
  ATTN_CHECK_CUDA(cudaStreamSynchronize(s));
  return l;
}

void Mlp::adam_step(float lr) {
  ++t;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<g1((int)NPARAM), 256, 0, ctx->stream>>>(params.as<float>(), grad.as<float>(), m.as<float>(),
                                                        v.as<float>(), (int)NPARAM, lr, b1, b2, 1e-8f, c1, c2);
  ctx->launches++;
}

void Mlp::init(attn_ctx* c, const float* host_params) {
  ctx = c;
  params.reserve(sizeof(float) * NPARAM);
  grad.reserve(sizeof(float) * NPARAM);
  m.reserve(sizeof(float) * NPARAM);
  v.reserve(sizeof(float) * NPARAM);
  ATTN_CHECK_CUDA(cudaMemcpyAsync(params.p, host_params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, ctx->stream));
  ATTN_CHECK_CUDA(cudaMemsetAsync(m.p, 0, sizeof(float) * NPARAM, ctx->stream));
  ATTN_CHECK_CUDA(cudaMemsetAsync(v.p, 0, sizeof(float) * NPARAM, ctx->stream));
  ATTN_CHECK_CUDA(cudaMemsetAsync(grad.p, 0, sizeof(float) * NPARAM, ctx->stream));
  t = 0;
}

}  // namespace attn
