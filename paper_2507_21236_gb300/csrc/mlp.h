// Learned disentangler initialiser: FP32 MLP state and kernels (internal).
#pragma once

#include "attn_internal.h"

namespace attn {

size_t mlp_param_count();

struct Mlp {
  attn_ctx* ctx = nullptr;
  DevBuf params, grad, m, v;                               // FP32 parameters and Adam moments
  DevBuf x, h1, h2, mo, u, gm, g2, g1b, lp, ut, xin;       // batch buffers
  int cap = 0;
  int t = 0;                                               // Adam step count
  void init(attn_ctx* c, const float* host_params);
  void ensure(int B);
  void upload_inputs(int B, const double* rho_host, const double* ut_host);
  void forward(int B);
  void predict(int B, const double* rho_host, double* u_host);
  float loss_grad(int B);
  void adam_step(float lr);
};

}  // namespace attn

struct attn_mlp {
  attn::Mlp net;
};
