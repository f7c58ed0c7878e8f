// The weight-predicting MLP of the learned smoother (no counterpart in the
// paper): 8 level features -> 64 -> 64 -> 4 weights of Eq. polsmootheropt,
//   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), o = W3 h2 + b3,
//   beta = beta_ref * exp(2 tanh(o / 2)),
// with forward, backward and Adam kernels in FP32.  Parameters are one vector
// [W1 (64x8), b1, W2 (64x64), b2, W3 (4x64), b3] (4996 floats).  Each sum over
// the batch is taken in sample order by one thread, so results repeat exactly.
#include "kernels_common.cuh"

namespace amgps {
namespace {

constexpr int NF = 8, NH = 64, NO = 4;
constexpr int OW1 = 0, OB1 = OW1 + NH * NF, OW2 = OB1 + NH, OB2 = OW2 + NH * NH,
              OW3 = OB2 + NH, OB3 = OW3 + NO * NH, NPARAM = OB3 + NO;
constexpr int NACT = NH + NH + NO;  // per sample: a1, a2, tanh(o / 2)
static_assert(NPARAM == 4996, "parameter layout");

// one block (64 threads) per sample
__global__ void __launch_bounds__(NH) k_mlp_forward(const float* __restrict__ th,
                                                    const float* __restrict__ F, int batch,
                                                    const float* __restrict__ ref,
                                                    float* __restrict__ beta,
                                                    float* __restrict__ acts) {
  const int b = blockIdx.x, j = threadIdx.x;
  if (b >= batch) return;
  __shared__ float f[NF], h1[NH], h2[NH];
  if (j < NF) f[j] = F[b * NF + j];
  __syncthreads();
  float a1 = th[OB1 + j];
  for (int i = 0; i < NF; ++i) a1 = fmaf(th[OW1 + j * NF + i], f[i], a1);
  h1[j] = fmaxf(a1, 0.f);
  __syncthreads();
  float a2 = th[OB2 + j];
  for (int i = 0; i < NH; ++i) a2 = fmaf(th[OW2 + j * NH + i], h1[i], a2);
  h2[j] = fmaxf(a2, 0.f);
  acts[b * NACT + j] = a1;
  acts[b * NACT + NH + j] = a2;
  __syncthreads();
  if (j < NO) {
    float o = th[OB3 + j];
    for (int i = 0; i < NH; ++i) o = fmaf(th[OW3 + j * NH + i], h2[i], o);
    const float t = tanhf(0.5f * o);
    acts[b * NACT + 2 * NH + j] = t;
    beta[b * NO + j] = ref[j] * expf(2.f * t);
  }
}

// per-sample deltas: go (4), ga2 (64), ga1 (64) into work[b * NACT + ...]
__global__ void __launch_bounds__(NH) k_mlp_deltas(const float* __restrict__ th,
                                                   const float* __restrict__ acts,
                                                   const float* __restrict__ beta,
                                                   const float* __restrict__ gbeta, int batch,
                                                   float* __restrict__ work) {
  const int b = blockIdx.x, j = threadIdx.x;
  if (b >= batch) return;
  __shared__ float go[NO], ga2[NH];
  if (j < NO) {
    const float t = acts[b * NACT + 2 * NH + j];
    go[j] = gbeta[b * NO + j] * beta[b * NO + j] * (1.f - t * t);  // d beta / d o
    work[b * NACT + 2 * NH + j] = go[j];
  }
  __syncthreads();
  float gh2 = 0.f;
  for (int q = 0; q < NO; ++q) gh2 = fmaf(th[OW3 + q * NH + j], go[q], gh2);
  const float g2 = acts[b * NACT + NH + j] > 0.f ? gh2 : 0.f;
  ga2[j] = g2;
  work[b * NACT + NH + j] = g2;
  __syncthreads();
  float gh1 = 0.f;
  for (int i = 0; i < NH; ++i) gh1 = fmaf(th[OW2 + i * NH + j], ga2[i], gh1);
  work[b * NACT + j] = acts[b * NACT + j] > 0.f ? gh1 : 0.f;
}

// parameter gradients: one thread per parameter, sum over samples in order
__global__ void __launch_bounds__(256) k_mlp_pgrad(const float* __restrict__ F,
                                                   const float* __restrict__ acts,
                                                   const float* __restrict__ work, int batch,
                                                   float* __restrict__ grads) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  float g = 0.f;
  if (p < OB1) {
    const int j = p / NF, i = p % NF;
    for (int b = 0; b < batch; ++b) g = fmaf(work[b * NACT + j], F[b * NF + i], g);
  } else if (p < OW2) {
    const int j = p - OB1;
    for (int b = 0; b < batch; ++b) g += work[b * NACT + j];
  } else if (p < OB2) {
    const int j = (p - OW2) / NH, i = (p - OW2) % NH;
    for (int b = 0; b < batch; ++b)
      g = fmaf(work[b * NACT + NH + j], fmaxf(acts[b * NACT + i], 0.f), g);
  } else if (p < OW3) {
    const int j = p - OB2;
    for (int b = 0; b < batch; ++b) g += work[b * NACT + NH + j];
  } else if (p < OB3) {
    const int q = (p - OW3) / NH, i = (p - OW3) % NH;
    for (int b = 0; b < batch; ++b)
      g = fmaf(work[b * NACT + 2 * NH + q], fmaxf(acts[b * NACT + NH + i], 0.f), g);
  } else {
    const int q = p - OB3;
    for (int b = 0; b < batch; ++b) g += work[b * NACT + 2 * NH + q];
  }
  grads[p] = g;
}

__global__ void __launch_bounds__(256) k_mlp_adam(float* __restrict__ th,
                                                  const float* __restrict__ g,
                                                  float* __restrict__ m, float* __restrict__ v,
                                                  float c1, float c2, float lr, float b1, float b2,
                                                  float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const float mi = b1 * m[p] + (1.f - b1) * g[p];
  const float vi = b2 * v[p] + (1.f - b2) * g[p] * g[p];
  m[p] = mi;
  v[p] = vi;
  th[p] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

void mlp_forward(const float* th, const float* F, int batch, const float* ref, float* beta,
                 float* acts, cudaStream_t s) {
  k_mlp_forward<<<batch, NH, 0, s>>>(th, F, batch, ref, beta, acts);
  count_launch();
}

void mlp_backward(const float* th, const float* F, const float* acts, const float* beta,
                  int batch, const float* gbeta, float* work, float* grads, cudaStream_t s) {
  k_mlp_deltas<<<batch, NH, 0, s>>>(th, acts, beta, gbeta, batch, work);
  count_launch();
  k_mlp_pgrad<<<(NPARAM + 255) / 256, 256, 0, s>>>(F, acts, work, batch, grads);
  count_launch();
}

void mlp_adam(float* th, const float* g, float* m, float* v, int step, float lr, float b1,
              float b2, float eps, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(th, g, m, v, c1, c2, lr, b1, b2, eps);
  count_launch();
}

}  // namespace amgps
