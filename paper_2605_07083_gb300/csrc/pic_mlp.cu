// pic_mlp.cu -- the surrogate MLP 5 -> 128 -> 128 -> 128 -> 4 (GELU hidden
// layers, linear output): fused forward+backward and fused reduce+Adam.
//
// Mixed precision: the forward and backward read bfloat16 weights (a copy of
// the FP32 master weights), FP32 biases, and keep FP32 activations and
// accumulators; the optimiser updates the FP32 master and re-rounds the
// bfloat16 copy.  Deterministic: per-CTA gradient partials are summed in a
// fixed order.  The network is tiny (34k parameters); these kernels are
// latency-bound by design and sit outside the particle hot path.
//
// Parameter layout (flat FP32 master, bfloat16 copy with the same indices):
// for each layer, W (n_out x n_in row-major) then b (n_out).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pic.h"

namespace pic {
namespace mlp {

constexpr int IN = 5, H = 128, OUT = 4;
constexpr int TILE = 32;                     // samples per CTA
constexpr int LD = H + 1;                    // padded row of an activation tile
constexpr int oW1 = 0, ob1 = oW1 + H * IN, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H,
              ob3 = oW3 + H * H, oW4 = ob3 + H, ob4 = oW4 + OUT * H, NP = ob4 + OUT;
static_assert(NP == PIC_MLP_PARAMS, "parameter count");

__device__ __forceinline__ float bf(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * __expf(-0.5f * x * x);
  return cdf + x * pdf;
}

struct Smem {
  float a0[TILE][IN];
  float z1[TILE][LD], a1[TILE][LD];
  float z2[TILE][LD], a2[TILE][LD];
  float z3[TILE][LD], a3[TILE][LD];
  float dy[TILE][OUT];
  float red[H];
};

// hidden layer: z[s][j] = b[j] + sum_k W[j][k] a[s][k], thread j = hidden unit
__device__ __forceinline__ void hidden(const __nv_bfloat16* W, const float* b, const float (*a)[LD],
                                       float (*z)[LD], float (*act)[LD], int n_in, int ns) {
  const int j = threadIdx.x;
  float acc[TILE];
#pragma unroll
  for (int s = 0; s < TILE; ++s) acc[s] = b[j];
  for (int k = 0; k < n_in; ++k) {
    const float w = bf(W, j * n_in + k);
#pragma unroll
    for (int s = 0; s < TILE; ++s) acc[s] = fmaf(w, a[s][k], acc[s]);
  }
#pragma unroll
  for (int s = 0; s < TILE; ++s) {
    if (s < ns) {
      z[s][j] = acc[s];
      act[s][j] = gelu(acc[s]);
    }
  }
}

// gW[j][k] = sum_s d[s][j] a[s][k]; thread j = output unit (row)
__device__ __forceinline__ void weight_grad(const float (*d)[LD], const float (*a)[LD], int n_in,
                                            int ns, float* gW, float* gb) {
  const int j = threadIdx.x;
  for (int k = 0; k < n_in; ++k) {
    float g = 0.0f;
    for (int s = 0; s < ns; ++s) g = fmaf(d[s][j], a[s][k], g);
    gW[j * n_in + k] = g;
  }
  float g = 0.0f;
  for (int s = 0; s < ns; ++s) g += d[s][j];
  gb[j] = g;
}

// delta of the layer below: out[s][k] = (sum_j W[j][k] d[s][j]) gelu'(z[s][k])
__device__ __forceinline__ void back_delta(const __nv_bfloat16* W, const float (*d)[LD],
                                           float (*z)[LD], int ns) {
  const int k = threadIdx.x;
  float acc[TILE];
#pragma unroll
  for (int s = 0; s < TILE; ++s) acc[s] = 0.0f;
  for (int j = 0; j < H; ++j) {
    const float w = bf(W, j * H + k);
#pragma unroll
    for (int s = 0; s < TILE; ++s) acc[s] = fmaf(w, d[s][j], acc[s]);
  }
  __syncthreads();                          // every thread has read d before z is overwritten
#pragma unroll
  for (int s = 0; s < TILE; ++s)
    if (s < ns) z[s][k] = acc[s] * gelu_grad(z[s][k]);
}

// One CTA = one tile of up to TILE samples.  t == nullptr: forward only.
// part: per-CTA gradient partials [gridDim.x][NP]; lpart: per-CTA sum of
// squared errors.
__global__ void __launch_bounds__(H) k_mlp_fwd_bwd(const float* __restrict__ master,
                                                   const __nv_bfloat16* __restrict__ w,
                                                   const float* __restrict__ x,
                                                   const float* __restrict__ t, long long batch,
                                                   float* __restrict__ y, float* __restrict__ part,
                                                   float* __restrict__ lpart) {
  extern __shared__ __align__(16) unsigned char raw[];
  Smem& S = *reinterpret_cast<Smem*>(raw);
  const int j = threadIdx.x;
  const long long s0 = (long long)blockIdx.x * TILE;
  const int ns = (int)min((long long)TILE, batch - s0);
  for (int i = j; i < TILE * IN; i += H) {
    const int s = i / IN, k = i - s * IN;
    S.a0[s][k] = s < ns ? x[(s0 + s) * IN + k] : 0.0f;
  }
  __syncthreads();
  // layer 1 (fan-in 5) reads a0 through the same helper via a padded view
  {
    float acc[TILE];
#pragma unroll
    for (int s = 0; s < TILE; ++s) acc[s] = master[ob1 + j];
    for (int k = 0; k < IN; ++k) {
      const float wv = bf(w, oW1 + j * IN + k);
#pragma unroll
      for (int s = 0; s < TILE; ++s) acc[s] = fmaf(wv, S.a0[s][k], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < TILE; ++s) {
      S.z1[s][j] = acc[s];
      S.a1[s][j] = gelu(acc[s]);
    }
  }
  __syncthreads();
  hidden(w + oW2, master + ob2, S.a1, S.z2, S.a2, H, TILE);
  __syncthreads();
  hidden(w + oW3, master + ob3, S.a2, S.z3, S.a3, H, TILE);
  __syncthreads();
  // output layer: thread (o, s) = (j / 32, j % 32)
  {
    const int o = j >> 5, s = j & 31;
    float acc = master[ob4 + o];
    for (int k = 0; k < H; ++k) acc = fmaf(bf(w, oW4 + o * H + k), S.a3[s][k], acc);
    if (s < ns) {
      if (y) y[(s0 + s) * OUT + o] = acc;
      float d = 0.0f, e2 = 0.0f;
      if (t) {
        const float diff = acc - t[(s0 + s) * OUT + o];
        d = 2.0f * diff / (float)(batch * OUT);
        e2 = diff * diff;
      }
      S.dy[s][o] = d;
      S.red[j] = e2;
    } else {
      S.dy[s][o] = 0.0f;
      S.red[j] = 0.0f;
    }
  }
  __syncthreads();
  if (!t) return;
  if (j < 32) {                              // loss partial, fixed order
    float v = S.red[j] + S.red[j + 32] + S.red[j + 64] + S.red[j + 96];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (j == 0) lpart[blockIdx.x] = v;
  }
  float* g = part + (size_t)blockIdx.x * NP;
  // output layer gradients: thread k = hidden unit
  {
    const int k = j;
    for (int o = 0; o < OUT; ++o) {
      float gw = 0.0f;
      for (int s = 0; s < ns; ++s) gw = fmaf(S.dy[s][o], S.a3[s][k], gw);
      g[oW4 + o * H + k] = gw;
    }
    if (k < OUT) {
      float gb = 0.0f;
      for (int s = 0; s < ns; ++s) gb += S.dy[s][k];
      g[ob4 + k] = gb;
    }
    // delta of layer 3: (sum_o W4[o][k] dy[s][o]) gelu'(z3[s][k]), kept in z3
    for (int s = 0; s < TILE; ++s) {
      float a = 0.0f;
      for (int o = 0; o < OUT; ++o) a = fmaf(bf(w, oW4 + o * H + k), S.dy[s][o], a);
      S.z3[s][k] = s < ns ? a * gelu_grad(S.z3[s][k]) : 0.0f;
    }
  }
  __syncthreads();
  weight_grad(S.z3, S.a2, H, ns, g + oW3, g + ob3);
  back_delta(w + oW3, S.z3, S.z2, ns);       // z2 <- delta of layer 2
  __syncthreads();
  weight_grad(S.z2, S.a1, H, ns, g + oW2, g + ob2);
  back_delta(w + oW2, S.z2, S.z1, ns);       // z1 <- delta of layer 1
  __syncthreads();
  {
    for (int k = 0; k < IN; ++k) {
      float gw = 0.0f;
      for (int s = 0; s < ns; ++s) gw = fmaf(S.z1[s][j], S.a0[s][k], gw);
      g[oW1 + j * IN + k] = gw;
    }
    float gb = 0.0f;
    for (int s = 0; s < ns; ++s) gb += S.z1[s][j];
    g[ob1 + j] = gb;
  }
}

// grad[p] = sum over CTAs of the partials (fixed order); optional Adam update
// of the FP32 master with the bfloat16 copy re-rounded (Kingma & Ba 2015).
__global__ void k_mlp_reduce_adam(const float* __restrict__ part, const float* __restrict__ lpart,
                                  int n_part, long long batch, float* __restrict__ grad,
                                  float* __restrict__ loss, float* __restrict__ master,
                                  __nv_bfloat16* __restrict__ w, float* __restrict__ m,
                                  float* __restrict__ v, float lr, float beta1, float beta2,
                                  float eps, float bc1, float bc2, int do_adam) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss) {
    float L = 0.0f;
    for (int b = 0; b < n_part; ++b) L += lpart[b];
    *loss = L / (float)(batch * OUT);
  }
  if (p >= NP) return;
  float gsum = 0.0f;
  for (int b = 0; b < n_part; ++b) gsum += part[(size_t)b * NP + p];
  if (grad) grad[p] = gsum;
  if (!do_adam) return;
  const float mm = beta1 * m[p] + (1.0f - beta1) * gsum;
  const float vv = beta2 * v[p] + (1.0f - beta2) * gsum * gsum;
  m[p] = mm;
  v[p] = vv;
  const float th = master[p] - lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
  master[p] = th;
  w[p] = __float2bfloat16_rn(th);
}

__global__ void k_mlp_cast(const float* __restrict__ master, __nv_bfloat16* __restrict__ w) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NP) w[p] = __float2bfloat16_rn(master[p]);
}

size_t scratch_floats(long long batch) {
  const long long nblk = (batch + TILE - 1) / TILE;
  return (size_t)nblk * NP + (size_t)nblk;
}

int launch_fwd_bwd(const float* master, const uint16_t* w, const float* x, const float* t,
                   long long batch, float* y, float* scratch, size_t scratch_bytes,
                   cudaStream_t s, int* nblk_out) {
  const long long nblk = (batch + TILE - 1) / TILE;
  if (t && scratch_bytes < scratch_floats(batch) * sizeof(float)) return PIC_EINVAL;
  static bool attr_done = false;
  if (!attr_done) {
    if (cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(Smem)) != cudaSuccess)
      return PIC_ECUDA;
    attr_done = true;
  }
  float* part = t ? scratch : nullptr;
  float* lpart = t ? scratch + (size_t)nblk * NP : nullptr;
  k_mlp_fwd_bwd<<<(unsigned)nblk, H, sizeof(Smem), s>>>(
      master, reinterpret_cast<const __nv_bfloat16*>(w), x, t, batch, y, part, lpart);
  if (nblk_out) *nblk_out = (int)nblk;
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

}  // namespace mlp
}  // namespace pic

using namespace pic::mlp;

extern "C" {

size_t pic_mlp_scratch_bytes(int64_t batch) {
  return batch > 0 ? pic::mlp::scratch_floats(batch) * sizeof(float) : 0;
}

int pic_mlp_cast_bf16(const float* master, uint16_t* w_bf16, void* stream) {
  if (!master || !w_bf16) return PIC_EINVAL;
  k_mlp_cast<<<(NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      master, reinterpret_cast<__nv_bfloat16*>(w_bf16));
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_mlp_forward(const float* master, const uint16_t* w_bf16, const float* x, int64_t batch,
                    float* y, void* stream) {
  if (!master || !w_bf16 || !x || !y || batch < 0) return PIC_EINVAL;
  if (batch == 0) return PIC_OK;
  return launch_fwd_bwd(master, w_bf16, x, nullptr, batch, y, nullptr, 0, (cudaStream_t)stream,
                        nullptr);
}

int pic_mlp_grad(const float* master, const uint16_t* w_bf16, const float* x, const float* t,
                 int64_t batch, float* grad, float* loss, float* scratch, size_t scratch_bytes,
                 void* stream) {
  if (!master || !w_bf16 || !x || !t || !grad || batch <= 0 || !scratch) return PIC_EINVAL;
  int nblk = 0;
  int rc = launch_fwd_bwd(master, w_bf16, x, t, batch, nullptr, scratch, scratch_bytes,
                          (cudaStream_t)stream, &nblk);
  if (rc != PIC_OK) return rc;
  k_mlp_reduce_adam<<<(NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      scratch, scratch + (size_t)nblk * NP, nblk, batch, grad, loss, nullptr, nullptr, nullptr,
      nullptr, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, 0);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_mlp_train_step(float* master, uint16_t* w_bf16, float* adam_m, float* adam_v,
                       int64_t step, float lr, float beta1, float beta2, float eps, const float* x,
                       const float* t, int64_t batch, float* loss, float* scratch,
                       size_t scratch_bytes, void* stream) {
  if (!master || !w_bf16 || !adam_m || !adam_v || !x || !t || batch <= 0 || step < 1 || !scratch)
    return PIC_EINVAL;
  int nblk = 0;
  int rc = launch_fwd_bwd(master, w_bf16, x, t, batch, nullptr, scratch, scratch_bytes,
                          (cudaStream_t)stream, &nblk);
  if (rc != PIC_OK) return rc;
  const float bc1 = 1.0f - powf(beta1, (float)step), bc2 = 1.0f - powf(beta2, (float)step);
  k_mlp_reduce_adam<<<(NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      scratch, scratch + (size_t)nblk * NP, nblk, batch, nullptr, loss, master,
      reinterpret_cast<__nv_bfloat16*>(w_bf16), adam_m, adam_v, lr, beta1, beta2, eps, bc1, bc2,
      1);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

}  // extern "C"
