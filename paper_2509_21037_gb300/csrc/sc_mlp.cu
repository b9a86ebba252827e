// Forward, backward and Adam kernels of the variant-predicting MLP
// (include/sc_mlp.h).  The network is tiny (tens of inputs, 64 hidden units,
// batches of thousands of subdomains), so each dense layer is one kernel with
// one thread per output element; the weight gradient reduces over the batch
// with one warp per weight row.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "sc_mlp.h"

namespace {

constexpr int kT = 256;

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

// out[b, o] = act(sum_i in[b, i] W[o, i] + bias[o])
__global__ void dense_fwd(const float *__restrict__ in, const float *__restrict__ W, const float *__restrict__ bias,
                          float *__restrict__ out, int B, int nin, int nout, int relu) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= (int64_t)B * nout) return;
  const int b = (int)(k / nout), o = (int)(k % nout);
  float s = bias[o];
  for (int i = 0; i < nin; ++i) s = fmaf(in[(int64_t)b * nin + i], W[(int64_t)o * nin + i], s);
  out[k] = relu ? fmaxf(s, 0.f) : s;
}

// dY = 2 mask (Y - T) / sum(mask); loss partials by atomics
__global__ void mse_grad(const float *__restrict__ Y, const float *__restrict__ T, const float *__restrict__ mask,
                         int64_t n, const float *__restrict__ inv_count, float *__restrict__ dY,
                         float *__restrict__ loss) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float l = 0.f;
  if (k < n) {
    const float d = (Y[k] - T[k]) * mask[k];
    dY[k] = 2.f * d * inv_count[0];
    l = d * d * inv_count[0];
  }
  for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

__global__ void mask_count(const float *__restrict__ mask, int64_t n, float *__restrict__ cnt) {
  float s = 0.f;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    s += mask[k];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(cnt, s);
}

__global__ void invert(float *x) { x[0] = x[0] > 0.f ? 1.f / x[0] : 0.f; }

// din[b, i] = (sum_o dout[b, o] W[o, i]) * (relu_of_in ? (in[b, i] > 0) : 1)
__global__ void dense_bwd_in(const float *__restrict__ dout, const float *__restrict__ W,
                             const float *__restrict__ in, float *__restrict__ din, int B, int nin, int nout,
                             int relu_of_in) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= (int64_t)B * nin) return;
  const int b = (int)(k / nin), i = (int)(k % nin);
  float s = 0.f;
  for (int o = 0; o < nout; ++o) s = fmaf(dout[(int64_t)b * nout + o], W[(int64_t)o * nin + i], s);
  if (relu_of_in && !(in[k] > 0.f)) s = 0.f;
  din[k] = s;
}

// dW[o, i] = sum_b dout[b, o] in[b, i]; db[o] = sum_b dout[b, o].  One warp
// per output unit o; lanes split the batch.
__global__ void dense_bwd_w(const float *__restrict__ dout, const float *__restrict__ in, float *__restrict__ dW,
                            float *__restrict__ db, int B, int nin, int nout) {
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= nout) return;
  const int o = warp;
  for (int i = -1; i < nin; ++i) {
    float s = 0.f;
    for (int b = lane; b < B; b += 32) s = fmaf(dout[(int64_t)b * nout + o], i < 0 ? 1.f : in[(int64_t)b * nin + i], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) {
      if (i < 0) db[o] = s;
      else dW[(int64_t)o * nin + i] = s;
    }
  }
}

__global__ void adam_kernel(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

struct Layout {
  int64_t w1, b1, w2, b2, w3, b3, total;
};

bool valid(const sc_mlp_shape *s) {
  return s && s->n_in > 0 && s->n_hidden > 0 && s->n_out > 0 && s->n_in <= 4096 && s->n_hidden <= 4096 &&
         s->n_out <= 4096;
}

Layout layout(const sc_mlp_shape &s) {
  Layout L;
  L.w1 = 0;
  L.b1 = L.w1 + (int64_t)s.n_hidden * s.n_in;
  L.w2 = L.b1 + s.n_hidden;
  L.b2 = L.w2 + (int64_t)s.n_hidden * s.n_hidden;
  L.w3 = L.b2 + s.n_hidden;
  L.b3 = L.w3 + (int64_t)s.n_out * s.n_hidden;
  L.total = L.b3 + s.n_out;
  return L;
}

// workspace: H1, H2 [B x H], Y [B x O], dY [B x O], dH2, dH1 [B x H], 2 scalars
struct Ws {
  float *H1, *H2, *Y, *dY, *dH2, *dH1, *scal;
};

Ws carve(const sc_mlp_shape &s, int B, float *ws) {
  Ws w;
  const int64_t bh = (int64_t)B * s.n_hidden, bo = (int64_t)B * s.n_out;
  w.H1 = ws;
  w.H2 = w.H1 + bh;
  w.Y = w.H2 + bh;
  w.dY = w.Y + bo;
  w.dH2 = w.dY + bo;
  w.dH1 = w.dH2 + bh;
  w.scal = w.dH1 + bh;
  return w;
}

void forward(const sc_mlp_shape &s, const Layout &L, const float *P, const float *X, int B, const Ws &w, float *Y,
             cudaStream_t st) {
  const int H = s.n_hidden, O = s.n_out;
  dense_fwd<<<blocks_for((int64_t)B * H), kT, 0, st>>>(X, P + L.w1, P + L.b1, w.H1, B, s.n_in, H, 1);
  dense_fwd<<<blocks_for((int64_t)B * H), kT, 0, st>>>(w.H1, P + L.w2, P + L.b2, w.H2, B, H, H, 1);
  dense_fwd<<<blocks_for((int64_t)B * O), kT, 0, st>>>(w.H2, P + L.w3, P + L.b3, Y, B, H, O, 0);
}

}  // namespace

extern "C" {

int64_t sc_mlp_param_count(const sc_mlp_shape *s) { return valid(s) ? layout(*s).total : -1; }

int64_t sc_mlp_workspace_floats(const sc_mlp_shape *s, int32_t batch) {
  if (!valid(s) || batch < 0) return -1;
  return 4 * (int64_t)batch * s->n_hidden + 2 * (int64_t)batch * s->n_out + 2;
}

int sc_mlp_forward(const sc_mlp_shape *s, const float *params, const float *X, int32_t batch, float *Y, float *ws,
                   void *stream) {
  if (!valid(s) || batch < 0 || (batch > 0 && (!params || !X || !Y || !ws))) return 1;
  if (batch == 0) return 0;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Layout L = layout(*s);
  const Ws w = carve(*s, batch, ws);
  forward(*s, L, params, X, batch, w, Y, st);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int sc_mlp_loss_grad(const sc_mlp_shape *s, const float *params, const float *X, const float *T, const float *mask,
                     int32_t batch, float *grads, float *loss, float *ws, void *stream) {
  if (!valid(s) || batch <= 0 || !params || !X || !T || !mask || !grads || !loss || !ws) return 1;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Layout L = layout(*s);
  const Ws w = carve(*s, batch, ws);
  const int H = s->n_hidden, O = s->n_out, B = batch;
  forward(*s, L, params, X, B, w, w.Y, st);
  if (cudaMemsetAsync(w.scal, 0, 2 * sizeof(float), st) != cudaSuccess) return 3;
  if (cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return 3;
  const int64_t nout = (int64_t)B * O;
  mask_count<<<blocks_for(nout) < 152u * 4 ? blocks_for(nout) : 152u * 4, kT, 0, st>>>(mask, nout, w.scal);
  invert<<<1, 1, 0, st>>>(w.scal);
  mse_grad<<<blocks_for(nout), kT, 0, st>>>(w.Y, T, mask, nout, w.scal, w.dY, loss);
  // layer 3
  dense_bwd_w<<<blocks_for(32LL * O), kT, 0, st>>>(w.dY, w.H2, grads + L.w3, grads + L.b3, B, H, O);
  dense_bwd_in<<<blocks_for((int64_t)B * H), kT, 0, st>>>(w.dY, params + L.w3, w.H2, w.dH2, B, H, O, 1);
  // layer 2
  dense_bwd_w<<<blocks_for(32LL * H), kT, 0, st>>>(w.dH2, w.H1, grads + L.w2, grads + L.b2, B, H, H);
  dense_bwd_in<<<blocks_for((int64_t)B * H), kT, 0, st>>>(w.dH2, params + L.w2, w.H1, w.dH1, B, H, H, 1);
  // layer 1
  dense_bwd_w<<<blocks_for(32LL * H), kT, 0, st>>>(w.dH1, X, grads + L.w1, grads + L.b1, B, s->n_in, H);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int sc_mlp_adam(int64_t n, float *params, const float *grads, float *m, float *v, float lr, float beta1, float beta2,
                float eps, int32_t step, void *stream) {
  if (n < 0 || step < 1 || (n > 0 && (!params || !grads || !m || !v))) return 1;
  if (n == 0) return 0;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  adam_kernel<<<blocks_for(n), kT, 0, static_cast<cudaStream_t>(stream)>>>(n, params, grads, m, v, lr, beta1, beta2,
                                                                          eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

}  // extern "C"
