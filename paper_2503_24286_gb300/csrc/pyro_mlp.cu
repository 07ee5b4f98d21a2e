// Learned initial guess for the Newton temperature solve: a small MLP
//   x (D = N+1 features: normalised e, Y_1..Y_N) -> 64 -> 64 -> 1 (SiLU), BF16
// weights and activations with FP32 accumulation, trained here by hand-written
// forward/backward/Adam kernels on states whose internal energy the library's
// own energy kernel computes from (T, Y).  The guess only seeds the FP64 Newton
// iteration (Sec. A.3.1 Eq. delta_temp), which still runs to the same
// tolerance, so results do not depend on the network.
//
// Parameter vector (FP32 master copy), row-major:
//   W1[H][D], b1[H], W2[H][H], b2[H], w3[H], b3
// Features: x_0 = bf16(float((e - e_mean) / e_std)), x_{1+k} = bf16(trunc32(Y_k) * N)
// (trunc32: truncation of the double to float; the factor N brings the mass
// fractions to O(1)).
// Network (the same rounding points as the inference kernel):
//   a1_o = bf16(silu(b1_o + sum_i bf16(W1_oi) x_i))
//   a2_o = bf16(silu(b2_o + sum_i bf16(W2_oi) a1_i))
//   y    = b3 + sum_i bf16(w3_i) a2_i,     T_guess = clip(T_mean + T_std y, 200, 3500)
// Training loss: mean squared error of y against t = (T - T_mean)/T_std; the
// roundings are treated as the identity in the backward pass.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <random>
#include <string>
#include <vector>

#include "pyro.h"
#include "pyro_internal.h"

namespace {

constexpr int H = 64;           // hidden width
constexpr int DMAX = 64;        // features (N + 1) supported by the learned guess
constexpr int SB = 64;          // samples per block in the training kernel
constexpr int TPB = 128;        // threads per block in the training kernel
constexpr size_t GRAD_SMEM = sizeof(float) * (H * DMAX + H * H + 3 * H + SB * (DMAX + 1) + 4 * SB * (H + 1) + SB);

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
// double -> float by truncating the mantissa (tiny values flush to zero)
__device__ __forceinline__ float trunc32(double x) {
  int h = __double2hiint(x);
  unsigned l = (unsigned)__double2loint(x);
  int e = ((h >> 20) & 0x7ff) - 896;
  unsigned sgn = (unsigned)h & 0x80000000u;
  unsigned bits = sgn | ((unsigned)e << 23) | (((unsigned)h & 0xfffffu) << 3) | (l >> 29);
  bits = (e <= 0) ? sgn : bits;
  bits = (e >= 255) ? (sgn | 0x7f800000u) : bits;
  return __uint_as_float(bits);
}
__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
  float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// sum and sum of squares of e and T (for the normalisation), in double
__global__ void mlp_stats_kernel(int64_t n, const double* __restrict__ e, const double* __restrict__ T,
                                 double* __restrict__ acc) {
  double se = 0, se2 = 0, st = 0, st2 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = e[i], b = T[i];
    se += a; se2 += a * a; st += b; st2 += b * b;
  }
  for (int o = 16; o > 0; o >>= 1) {
    se += __shfl_down_sync(0xffffffffu, se, o);
    se2 += __shfl_down_sync(0xffffffffu, se2, o);
    st += __shfl_down_sync(0xffffffffu, st, o);
    st2 += __shfl_down_sync(0xffffffffu, st2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc + 0, se); atomicAdd(acc + 1, se2); atomicAdd(acc + 2, st); atomicAdd(acc + 3, st2);
  }
}

// One minibatch: forward + backward of SB samples per block; gradients of the
// whole batch accumulate (scaled by 1/B) into grad[] with atomics; the batch's
// squared error accumulates into loss[0].
__global__ void __launch_bounds__(TPB) mlp_grad_kernel(int64_t n, int64_t start, int B, int N,
    const double* __restrict__ e, const double* __restrict__ Y, const double* __restrict__ T,
    const float* __restrict__ P, const float* __restrict__ norm, float* __restrict__ grad,
    double* __restrict__ loss) {
  const int D = N + 1;
  extern __shared__ float smem[];
  float* sW1 = smem;                    // [H * DMAX] bf16-rounded weights as float
  float* sW2 = sW1 + H * DMAX;          // [H * H]
  float* sb1 = sW2 + H * H;             // [H]
  float* sb2 = sb1 + H;
  float* sw3 = sb2 + H;
  float (*sX)[DMAX + 1] = (float (*)[DMAX + 1])(sw3 + H);          // [SB][DMAX+1]
  float (*sZ1)[H + 1] = (float (*)[H + 1])((float*)sX + SB * (DMAX + 1));
  float (*sA1)[H + 1] = sZ1 + SB;
  float (*sZ2)[H + 1] = sA1 + SB;
  float (*sA2)[H + 1] = sZ2 + SB;
  float* sdy = (float*)(sA2 + SB);      // [SB]
  const float* W1 = P;
  const float* b1 = W1 + H * D;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* w3 = b2 + H;
  const float b3 = w3[H];
  for (int i = threadIdx.x; i < H * D; i += TPB) sW1[i] = bfr(W1[i]);
  for (int i = threadIdx.x; i < H * H; i += TPB) sW2[i] = bfr(W2[i]);
  for (int i = threadIdx.x; i < H; i += TPB) { sb1[i] = b1[i]; sb2[i] = b2[i]; sw3[i] = bfr(w3[i]); }
  const float e_mean = norm[0], e_inv = 1.0f / norm[1], T_mean = norm[2], T_inv = 1.0f / norm[3];
  const int64_t s0 = start + (int64_t)blockIdx.x * SB;
  // features
  for (int q = threadIdx.x; q < SB * D; q += TPB) {
    int s = q / D, i = q % D;
    int64_t idx = s0 + s;
    float v = 0.0f;
    if (idx < start + B && idx < n)
      v = i == 0 ? (float)((e[idx] - (double)e_mean) * (double)e_inv) : trunc32(Y[(int64_t)(i - 1) * n + idx]) * (float)N;
    sX[s][i] = bfr(v);
  }
  __syncthreads();
  // layer 1 and 2 (thread pairs split the outputs of one sample)
  for (int q = threadIdx.x; q < SB * H; q += TPB) {
    int s = q / H, o = q % H;
    float z = sb1[o];
    for (int i = 0; i < D; ++i) z = fmaf(sW1[o * D + i], sX[s][i], z);
    sZ1[s][o] = z;
    sA1[s][o] = bfr(silu_f(z));
  }
  __syncthreads();
  for (int q = threadIdx.x; q < SB * H; q += TPB) {
    int s = q / H, o = q % H;
    float z = sb2[o];
    for (int i = 0; i < H; ++i) z = fmaf(sW2[o * H + i], sA1[s][i], z);
    sZ2[s][o] = z;
    sA2[s][o] = bfr(silu_f(z));
  }
  __syncthreads();
  const float invB = 1.0f / (float)B;
  if (threadIdx.x < SB) {
    int s = threadIdx.x;
    int64_t idx = s0 + s;
    float dy = 0.0f;
    if (idx < start + B && idx < n) {
      float y = b3;
      for (int i = 0; i < H; ++i) y = fmaf(sw3[i], sA2[s][i], y);
      float t = (float)((T[idx] - (double)T_mean) * (double)T_inv);
      float r = y - t;
      atomicAdd(loss, (double)r * (double)r);
      dy = 2.0f * r * invB;
    }
    sdy[s] = dy;
  }
  __syncthreads();
  // delta2 = dy * w3 * silu'(z2)  (stored over Z2), delta1 = (W2^T delta2) * silu'(z1) (over Z1)
  for (int q = threadIdx.x; q < SB * H; q += TPB) {
    int s = q / H, o = q % H;
    sZ2[s][o] = sdy[s] * sw3[o] * dsilu_f(sZ2[s][o]);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < SB * H; q += TPB) {
    int s = q / H, i = q % H;
    float acc = 0.0f;
    for (int o = 0; o < H; ++o) acc = fmaf(sW2[o * H + i], sZ2[s][o], acc);
    sZ1[s][i] = acc * dsilu_f(sZ1[s][i]);
  }
  __syncthreads();
  float* gW1 = grad;
  float* gb1 = gW1 + H * D;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + H * H;
  float* gw3 = gb2 + H;
  float* gb3 = gw3 + H;
  for (int q = threadIdx.x; q < H * D; q += TPB) {
    int o = q / D, i = q % D;
    float acc = 0.0f;
    for (int s = 0; s < SB; ++s) acc = fmaf(sZ1[s][o], sX[s][i], acc);
    atomicAdd(gW1 + q, acc);
  }
  for (int q = threadIdx.x; q < H * H; q += TPB) {
    int o = q / H, i = q % H;
    float acc = 0.0f;
    for (int s = 0; s < SB; ++s) acc = fmaf(sZ2[s][o], sA1[s][i], acc);
    atomicAdd(gW2 + q, acc);
  }
  for (int o = threadIdx.x; o < H; o += TPB) {
    float a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    for (int s = 0; s < SB; ++s) { a1 += sZ1[s][o]; a2 += sZ2[s][o]; a3 = fmaf(sdy[s], sA2[s][o], a3); }
    atomicAdd(gb1 + o, a1);
    atomicAdd(gb2 + o, a2);
    atomicAdd(gw3 + o, a3);
  }
  if (threadIdx.x == 0) {
    float a = 0.0f;
    for (int s = 0; s < SB; ++s) a += sdy[s];
    atomicAdd(gb3, a);
  }
}

// Adam step on the FP32 master parameters; clears the gradient; refreshes the bf16 copy.
__global__ void mlp_adam_kernel(int P, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                                float* __restrict__ g, __nv_bfloat16* __restrict__ pb, float lr, float b1,
                                float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi; v[i] = vi; g[i] = 0.0f;
    float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void mlp_bf16_kernel(int P, const float* __restrict__ p, __nv_bfloat16* __restrict__ pb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) pb[i] = __float2bfloat16_rn(p[i]);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side (libpyro internals used by the runtime's C entry points)
// ---------------------------------------------------------------------------
namespace pyro {

int mlp_n_params(int D) { return H * D + H + H * H + H + H + 1; }

struct MlpState {
  int D = 0, P = 0;
  float* d_p = nullptr;            // FP32 master parameters
  float* d_m = nullptr;            // Adam moments
  float* d_v = nullptr;
  float* d_g = nullptr;            // gradient accumulator
  __nv_bfloat16* d_pb = nullptr;   // bf16 copy used by the inference kernel
  float* d_norm = nullptr;         // e_mean, e_std, T_mean, T_std
  double* d_acc = nullptr;         // reductions (loss, statistics)
  float h_norm[4] = {0, 1, 1200, 1};
  bool trained = false;
};

static int cuda_fail(const char* what, cudaError_t e) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return internal_fail(PYRO_ECUDA, m.c_str());
}

void mlp_free(MlpState* s) {
  if (!s) return;
  cudaFree(s->d_p); cudaFree(s->d_m); cudaFree(s->d_v); cudaFree(s->d_g); cudaFree(s->d_pb);
  cudaFree(s->d_norm); cudaFree(s->d_acc);
  delete s;
}

int mlp_create(int D, MlpState** out) {
  if (D > DMAX) return internal_fail(PYRO_EINVAL, "the learned guess supports at most 63 species");
  auto* s = new MlpState();
  s->D = D;
  s->P = mlp_n_params(D);
  size_t b = s->P * sizeof(float);
  cudaError_t e;
  if ((e = cudaMalloc(&s->d_p, b)) || (e = cudaMalloc(&s->d_m, b)) || (e = cudaMalloc(&s->d_v, b)) ||
      (e = cudaMalloc(&s->d_g, b)) || (e = cudaMalloc(&s->d_pb, s->P * sizeof(__nv_bfloat16))) ||
      (e = cudaMalloc(&s->d_norm, 4 * sizeof(float))) || (e = cudaMalloc(&s->d_acc, 8 * sizeof(double)))) {
    mlp_free(s);
    return cuda_fail("MLP allocation", e);
  }
  if ((e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRAD_SMEM))) {
    mlp_free(s);
    return cuda_fail("MLP kernel shared memory", e);
  }
  *out = s;
  return PYRO_OK;
}

// host parameter upload: FP64 values (packed as documented) + normalisation
int mlp_set(MlpState* s, const double* params, const double* norm4) {
  std::vector<float> h(s->P);
  for (int i = 0; i < s->P; ++i) h[i] = (float)params[i];
  for (int i = 0; i < 4; ++i) s->h_norm[i] = (float)norm4[i];
  cudaError_t e;
  if ((e = cudaMemcpy(s->d_p, h.data(), s->P * sizeof(float), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(s->d_norm, s->h_norm, 4 * sizeof(float), cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(s->d_m, 0, s->P * sizeof(float))) || (e = cudaMemset(s->d_v, 0, s->P * sizeof(float))) ||
      (e = cudaMemset(s->d_g, 0, s->P * sizeof(float))))
    return cuda_fail("MLP upload", e);
  mlp_bf16_kernel<<<(s->P + 255) / 256, 256>>>(s->P, s->d_p, s->d_pb);
  if ((e = cudaDeviceSynchronize())) return cuda_fail("MLP upload", e);
  s->trained = true;
  return PYRO_OK;
}

int mlp_get(MlpState* s, double* params, double* norm4) {
  std::vector<float> h(s->P);
  cudaError_t e = cudaMemcpy(h.data(), s->d_p, s->P * sizeof(float), cudaMemcpyDeviceToHost);
  if (e) return cuda_fail("MLP download", e);
  if (params) for (int i = 0; i < s->P; ++i) params[i] = h[i];
  if (norm4) for (int i = 0; i < 4; ++i) norm4[i] = s->h_norm[i];
  return PYRO_OK;
}

const void* mlp_device_bf16(const MlpState* s) { return s->d_pb; }
const float* mlp_device_params(const MlpState* s) { return s->d_p; }
const float* mlp_host_norm(const MlpState* s) { return s->h_norm; }
bool mlp_ready(const MlpState* s) { return s && s->trained; }

// Loss and gradient of a batch [start, start+B) (diagnostic / parity with the CPU model)
int mlp_grad(MlpState* s, int64_t n, int64_t start, int B, int N, const double* e, const double* Y,
             const double* T, double* loss_out, double* grad_out, cudaStream_t st) {
  cudaError_t err;
  if ((err = cudaMemsetAsync(s->d_g, 0, s->P * sizeof(float), st)) ||
      (err = cudaMemsetAsync(s->d_acc, 0, sizeof(double), st)))
    return cuda_fail("MLP gradient", err);
  int blocks = (B + SB - 1) / SB;
  mlp_grad_kernel<<<blocks, TPB, GRAD_SMEM, st>>>(n, start, B, N, e, Y, T, s->d_p, s->d_norm, s->d_g, s->d_acc);
  std::vector<float> g(s->P);
  double loss = 0;
  if ((err = cudaMemcpyAsync(g.data(), s->d_g, s->P * sizeof(float), cudaMemcpyDeviceToHost, st)) ||
      (err = cudaMemcpyAsync(&loss, s->d_acc, sizeof(double), cudaMemcpyDeviceToHost, st)) ||
      (err = cudaStreamSynchronize(st)))
    return cuda_fail("MLP gradient", err);
  if (grad_out) for (int i = 0; i < s->P; ++i) grad_out[i] = g[i];
  if (loss_out) *loss_out = loss / B;
  cudaMemsetAsync(s->d_g, 0, s->P * sizeof(float), st);
  return PYRO_OK;
}

// Initialise (seeded), normalise on the data, and train with Adam.
int mlp_train(MlpState* s, int64_t n, int N, const double* e, const double* Y, const double* T, int epochs,
              int batch, double lr, unsigned seed, double* final_loss, cudaStream_t st) {
  const int D = s->D;
  cudaError_t err;
  // normalisation from the data
  if ((err = cudaMemsetAsync(s->d_acc, 0, 8 * sizeof(double), st))) return cuda_fail("MLP statistics", err);
  mlp_stats_kernel<<<1216, 256, 0, st>>>(n, e, T, s->d_acc);
  double acc[4];
  if ((err = cudaMemcpyAsync(acc, s->d_acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st)) ||
      (err = cudaStreamSynchronize(st)))
    return cuda_fail("MLP statistics", err);
  double em = acc[0] / n, es = std::sqrt(std::max(acc[1] / n - em * em, 1e-300));
  double tm = acc[2] / n, ts = std::sqrt(std::max(acc[3] / n - tm * tm, 1e-300));
  double norm[4] = {em, es, tm, ts};
  // seeded initialisation: U(-1/sqrt(fan_in), 1/sqrt(fan_in)), zero biases
  std::vector<double> p0(s->P, 0.0);
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  for (int i = 0; i < H * D; ++i) p0[i] = u(rng) / std::sqrt((double)D);
  double* W2 = p0.data() + H * D + H;
  for (int i = 0; i < H * H; ++i) W2[i] = u(rng) / std::sqrt((double)H);
  double* w3 = W2 + H * H + H;
  for (int i = 0; i < H; ++i) w3[i] = u(rng) / std::sqrt((double)H);
  if (int rc = mlp_set(s, p0.data(), norm)) return rc;
  int64_t steps_per_epoch = n / batch;
  if (steps_per_epoch < 1) return internal_fail(PYRO_EINVAL, "fewer training states than one batch");
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  int64_t step = 0, total = steps_per_epoch * epochs;
  double last = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t k = 0; k < steps_per_epoch; ++k, ++step) {
      if (k == steps_per_epoch - 1 && ep == epochs - 1) cudaMemsetAsync(s->d_acc, 0, sizeof(double), st);
      mlp_grad_kernel<<<(batch + SB - 1) / SB, TPB, GRAD_SMEM, st>>>(n, k * batch, batch, N, e, Y, T, s->d_p, s->d_norm,
                                                             s->d_g, s->d_acc);
      // cosine-decayed learning rate
      double frac = (double)step / (double)total;
      float lr_t = (float)(lr * 0.5 * (1.0 + std::cos(3.14159265358979323846 * frac)));
      float c1 = 1.0f / (1.0f - std::pow(b1, (float)(step + 1)));
      float c2 = 1.0f / (1.0f - std::pow(b2, (float)(step + 1)));
      mlp_adam_kernel<<<(s->P + 255) / 256, 256, 0, st>>>(s->P, s->d_p, s->d_m, s->d_v, s->d_g, s->d_pb, lr_t, b1, b2,
                                                          eps, c1, c2);
    }
  }
  if ((err = cudaMemcpyAsync(&last, s->d_acc, sizeof(double), cudaMemcpyDeviceToHost, st)) ||
      (err = cudaStreamSynchronize(st)))
    return cuda_fail("MLP training", err);
  if (final_loss) *final_loss = last / batch;
  s->trained = true;
  return PYRO_OK;
}

// versioned binary: magic, version, D, P, norm[4] (double), params (float)
int mlp_save(const MlpState* s, const char* path) {
  std::vector<float> h(s->P);
  cudaError_t e = cudaMemcpy(h.data(), s->d_p, s->P * sizeof(float), cudaMemcpyDeviceToHost);
  if (e) return cuda_fail("MLP save", e);
  std::ofstream f(path, std::ios::binary);
  if (!f) return internal_fail(PYRO_EINVAL, "cannot write the MLP file");
  const char magic[8] = {'P', 'Y', 'R', 'O', 'M', 'L', 'P', '1'};
  int32_t hdr[2] = {s->D, s->P};
  double nm[4] = {s->h_norm[0], s->h_norm[1], s->h_norm[2], s->h_norm[3]};
  f.write(magic, 8); f.write((const char*)hdr, sizeof hdr); f.write((const char*)nm, sizeof nm);
  f.write((const char*)h.data(), h.size() * sizeof(float));
  return f ? PYRO_OK : internal_fail(PYRO_EINVAL, "short write of the MLP file");
}

int mlp_load(MlpState* s, const char* path) {
  std::ifstream f(path, std::ios::binary);
  if (!f) return internal_fail(PYRO_EINVAL, "cannot read the MLP file");
  char magic[8];
  int32_t hdr[2];
  double nm[4];
  f.read(magic, 8); f.read((char*)hdr, sizeof hdr); f.read((char*)nm, sizeof nm);
  if (!f || std::memcmp(magic, "PYROMLP1", 8) != 0) return internal_fail(PYRO_EINVAL, "not a PYROMLP1 file");
  if (hdr[0] != s->D || hdr[1] != s->P) return internal_fail(PYRO_EINVAL, "MLP file was trained for another species count");
  std::vector<float> h(s->P);
  f.read((char*)h.data(), h.size() * sizeof(float));
  if (!f) return internal_fail(PYRO_EINVAL, "short MLP file");
  std::vector<double> p(h.begin(), h.end());
  return mlp_set(s, p.data(), nm);
}

}  // namespace pyro
