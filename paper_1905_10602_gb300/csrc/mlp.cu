// Rank predictor: a small MLP (9 -> 64 -> 64 -> 64 -> 1, ReLU, FP32) that maps
// a recompression event's geometry (cell centre, size, level, offset to the
// eliminated neighbour) and log10(eps) to the truncation rank / 64.  Forward,
// backward and Adam kernels are written here; training runs on the GPU on the
// ranks that the SVD-mode factorization chose.
//
// Weight layout (floats, row-major W[in][out]): W1[9][64] b1[64] W2[64][64] b2[64]
// W3[64][64] b3[64] W4[64][1] b4[1]  -- IFMM_MLP_NWEIGHTS = 9025.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "common.h"
#include "mlp.h"

namespace ifmm {

static const int kIn = IFMM_MLP_IN, kH = 64;
static const int kDims[5] = {kIn, kH, kH, kH, 1};

// offsets of W_l and b_l in the flat weight vector
static void layer_offsets(int l, int* w, int* b) {
  int o = 0;
  for (int q = 0; q < l; ++q) o += kDims[q] * kDims[q + 1] + kDims[q + 1];
  *w = o;
  *b = o + kDims[l] * kDims[l + 1];
}

// out[s][j] = act(sum_i in[s][i] W[i][j] + b[j]); a thread per (sample, unit)
__global__ void k_mlp_layer(const float* __restrict__ in, int din, const float* __restrict__ W,
                            const float* __restrict__ b, float* __restrict__ out, int dout, int ns, int relu) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)ns * dout) return;
  const int s = (int)(e / dout), j = (int)(e % dout);
  float acc = b[j];
  const float* x = in + (long)s * din;
  for (int i = 0; i < din; ++i) acc = fmaf(x[i], W[i * dout + j], acc);
  out[e] = relu ? fmaxf(acc, 0.f) : acc;
}

// dL/dy for L = mean (y - t)^2 / 2, plus per-sample squared errors
__global__ void k_mlp_loss(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                           float* __restrict__ sq, int ns) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const float d = y[s] - t[s];
  dy[s] = d / (float)ns;
  sq[s] = 0.5f * d * d;
}

// din[s][i] = (sum_j dout[s][j] W[i][j]) * relu'(in[s][i])
__global__ void k_mlp_back_in(const float* __restrict__ dout, int dout_n, const float* __restrict__ W,
                              const float* __restrict__ act_in, float* __restrict__ din, int din_n, int ns) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)ns * din_n) return;
  const int s = (int)(e / din_n), i = (int)(e % din_n);
  float acc = 0.f;
  const float* g = dout + (long)s * dout_n;
  for (int j = 0; j < dout_n; ++j) acc = fmaf(g[j], W[i * dout_n + j], acc);
  din[e] = act_in[e] > 0.f ? acc : 0.f;
}

// dW[i][j] = sum_s in[s][i] dout[s][j]; db[j] = sum_s dout[s][j]: a thread per
// weight, summing over the samples in a fixed order (deterministic)
__global__ void k_mlp_back_w(const float* __restrict__ in, int din, const float* __restrict__ dout, int dn,
                             float* __restrict__ dW, float* __restrict__ db, int ns) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < din * dn) {
    const int i = e / dn, j = e % dn;
    double acc = 0.0;
    for (int s = 0; s < ns; ++s) acc += (double)in[(long)s * din + i] * (double)dout[(long)s * dn + j];
    dW[e] = (float)acc;
  } else if (e < din * dn + dn) {
    const int j = e - din * dn;
    double acc = 0.0;
    for (int s = 0; s < ns; ++s) acc += (double)dout[(long)s * dn + j];
    db[j] = (float)acc;
  }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// w -= lr * mhat / (sqrt(vhat) + 1e-8)
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float b1 = 0.9f, b2 = 0.999f;
  m[i] = b1 * m[i] + (1.f - b1) * g[i];
  v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  const float mh = m[i] / c1, vh = v[i] / c2;
  w[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// counter-based initialisation: SplitMix64 (Steele, Lea, Flood) of (seed, index)
// -> uniform in [-a, a]
__global__ void k_mlp_init(float* __restrict__ w, int n, unsigned long long seed, float a, int first, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(first + i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  const float u = (float)((z >> 40) * (1.0 / 16777216.0));  // [0, 1)
  w[first + i] = a * (2.f * u - 1.f);
  (void)n;
}

struct MlpBuffers {
  float* act[5] = {nullptr};   // activations per layer (act[0] = input)
  float* grad[5] = {nullptr};  // gradients w.r.t. activations
  float* sq = nullptr;
  int ns = 0;
  std::vector<float*> owned;
  float* get(size_t n) {
    float* p = nullptr;
    CKM(cudaMalloc(&p, sizeof(float) * std::max<size_t>(n, 1)));
    owned.push_back(p);
    return p;
  }
  MlpBuffers(int n) : ns(n) {
    for (int l = 0; l < 5; ++l) {
      act[l] = get((size_t)n * kDims[l]);
      grad[l] = get((size_t)n * kDims[l]);
    }
    sq = get(n);
  }
  // forward only: input and output in place, the hidden activations in work
  MlpBuffers(int n, const float* x, float* y, float* work) : ns(n) {
    act[0] = const_cast<float*>(x);
    for (int l = 1; l < 4; ++l) {
      act[l] = work;
      work += (size_t)n * kDims[l];
    }
    act[4] = y;
  }
  ~MlpBuffers() {
    for (auto p : owned) cudaFree(p);
  }
};

// forward over ns samples already in B.act[0]; result in B.act[4]
static void mlp_forward(const float* w, MlpBuffers& B, int ns, cudaStream_t s) {
  for (int l = 0; l < 4; ++l) {
    int wo, bo;
    layer_offsets(l, &wo, &bo);
    const long tot = (long)ns * kDims[l + 1];
    k_mlp_layer<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(B.act[l], kDims[l], w + wo, w + bo, B.act[l + 1],
                                                              kDims[l + 1], ns, l < 3);
  }
}

// loss and gradient (into g, IFMM_MLP_NWEIGHTS floats) for targets t
static void mlp_backward(const float* w, const float* t, float* g, MlpBuffers& B, int ns, cudaStream_t s) {
  k_mlp_loss<<<(ns + 255) / 256, 256, 0, s>>>(B.act[4], t, B.grad[4], B.sq, ns);
  for (int l = 3; l >= 0; --l) {
    int wo, bo;
    layer_offsets(l, &wo, &bo);
    const int nw = kDims[l] * kDims[l + 1] + kDims[l + 1];
    k_mlp_back_w<<<(nw + 255) / 256, 256, 0, s>>>(B.act[l], kDims[l], B.grad[l + 1], kDims[l + 1], g + wo, g + bo, ns);
    if (l > 0) {
      const long tot = (long)ns * kDims[l];
      k_mlp_back_in<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(B.grad[l + 1], kDims[l + 1], w + wo, B.act[l],
                                                                 B.grad[l], kDims[l], ns);
    }
  }
}

size_t mlp_predict_floats(int ns) { return (size_t)std::max(ns, 1) * (kDims[1] + kDims[2] + kDims[3]); }

void mlp_predict_device(const float* d_w, const float* d_x, float* d_y, int ns, cudaStream_t s, float* work) {
  if (ns <= 0) return;
  MlpBuffers B(ns, d_x, d_y, work);
  mlp_forward(d_w, B, ns, s);
}

}  // namespace ifmm

using namespace ifmm;

extern "C" {

ifmm_status ifmm_mlp_forward(const float* weights, const float* x, int64_t n, float* y, void* stream) {
  try {
    IFMM_REQUIRE(weights && x && y && n >= 0 && n < (1 << 26), IFMM_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    MlpBuffers B((int)std::max<int64_t>(n, 1));
    float* dw = B.get(IFMM_MLP_NWEIGHTS);
    CKM(cudaMemcpyAsync(dw, weights, sizeof(float) * IFMM_MLP_NWEIGHTS, cudaMemcpyHostToDevice, s));
    CKM(cudaMemcpyAsync(B.act[0], x, sizeof(float) * n * kIn, cudaMemcpyHostToDevice, s));
    mlp_forward(dw, B, (int)n, s);
    CKM(cudaMemcpyAsync(y, B.act[4], sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    CKM(cudaStreamSynchronize(s));
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

ifmm_status ifmm_mlp_grad(const float* weights, const float* x, const float* t, int64_t n, float* grad, float* loss,
                          void* stream) {
  try {
    IFMM_REQUIRE(weights && x && t && grad && n >= 1 && n < (1 << 26), IFMM_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    MlpBuffers B((int)n);
    float* dw = B.get(IFMM_MLP_NWEIGHTS);
    float* dg = B.get(IFMM_MLP_NWEIGHTS);
    float* dt = B.get(n);
    CKM(cudaMemcpyAsync(dw, weights, sizeof(float) * IFMM_MLP_NWEIGHTS, cudaMemcpyHostToDevice, s));
    CKM(cudaMemcpyAsync(B.act[0], x, sizeof(float) * n * kIn, cudaMemcpyHostToDevice, s));
    CKM(cudaMemcpyAsync(dt, t, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    mlp_forward(dw, B, (int)n, s);
    mlp_backward(dw, dt, dg, B, (int)n, s);
    std::vector<float> sq(n);
    CKM(cudaMemcpyAsync(grad, dg, sizeof(float) * IFMM_MLP_NWEIGHTS, cudaMemcpyDeviceToHost, s));
    CKM(cudaMemcpyAsync(sq.data(), B.sq, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    CKM(cudaStreamSynchronize(s));
    if (loss) {
      double acc = 0;
      for (float v : sq) acc += v;
      *loss = (float)(acc / (double)n);
    }
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

ifmm_status ifmm_mlp_train(const float* x, const float* t, int64_t n, int epochs, int batch, float lr, uint64_t seed,
                           float* weights, float* final_loss, void* stream) {
  try {
    IFMM_REQUIRE(x && t && weights && n >= 1 && n < (1 << 26) && epochs >= 1 && batch >= 1, IFMM_EINVAL,
                 "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int bs = (int)std::min<int64_t>(batch, n);
    MlpBuffers B(bs);
    float* dw = B.get(IFMM_MLP_NWEIGHTS);
    float* dg = B.get(IFMM_MLP_NWEIGHTS);
    float* dm = B.get(IFMM_MLP_NWEIGHTS);
    float* dv = B.get(IFMM_MLP_NWEIGHTS);
    float* dx = B.get((size_t)n * kIn);
    float* dt = B.get(n);
    CKM(cudaMemcpyAsync(dx, x, sizeof(float) * n * kIn, cudaMemcpyHostToDevice, s));
    CKM(cudaMemcpyAsync(dt, t, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    CKM(cudaMemsetAsync(dm, 0, sizeof(float) * IFMM_MLP_NWEIGHTS, s));
    CKM(cudaMemsetAsync(dv, 0, sizeof(float) * IFMM_MLP_NWEIGHTS, s));
    // He-uniform weights, zero biases
    CKM(cudaMemsetAsync(dw, 0, sizeof(float) * IFMM_MLP_NWEIGHTS, s));
    for (int l = 0; l < 4; ++l) {
      int wo, bo;
      layer_offsets(l, &wo, &bo);
      const int cnt = kDims[l] * kDims[l + 1];
      const float a = std::sqrt(6.0f / (float)kDims[l]);
      k_mlp_init<<<(cnt + 255) / 256, 256, 0, s>>>(dw, IFMM_MLP_NWEIGHTS, (unsigned long long)seed, a, wo, cnt);
    }
    long step = 0;
    const int nb = (int)((n + bs - 1) / bs);
    for (int ep = 0; ep < epochs; ++ep)
      for (int bi = 0; bi < nb; ++bi) {
        const int off = bi * bs;
        const int cur = (int)std::min<int64_t>(bs, n - off);
        CKM(cudaMemcpyAsync(B.act[0], dx + (long)off * kIn, sizeof(float) * cur * kIn, cudaMemcpyDeviceToDevice, s));
        mlp_forward(dw, B, cur, s);
        mlp_backward(dw, dt + off, dg, B, cur, s);
        ++step;
        const float c1 = 1.f - std::pow(0.9f, (float)step), c2 = 1.f - std::pow(0.999f, (float)step);
        k_adam<<<(IFMM_MLP_NWEIGHTS + 255) / 256, 256, 0, s>>>(dw, dg, dm, dv, IFMM_MLP_NWEIGHTS, lr, c1, c2);
      }
    CKM(cudaGetLastError());
    CKM(cudaMemcpyAsync(weights, dw, sizeof(float) * IFMM_MLP_NWEIGHTS, cudaMemcpyDeviceToHost, s));
    CKM(cudaStreamSynchronize(s));
    if (final_loss) {
      // loss over the whole set with the final weights
      MlpBuffers E((int)n);
      CKM(cudaMemcpyAsync(E.act[0], dx, sizeof(float) * n * kIn, cudaMemcpyDeviceToDevice, s));
      mlp_forward(dw, E, (int)n, s);
      float* g2 = E.get(IFMM_MLP_NWEIGHTS);
      mlp_backward(dw, dt, g2, E, (int)n, s);
      std::vector<float> sq(n);
      CKM(cudaMemcpyAsync(sq.data(), E.sq, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
      CKM(cudaStreamSynchronize(s));
      double acc = 0;
      for (float v : sq) acc += v;
      *final_loss = (float)(acc / (double)n);
    }
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

}  // extern "C"
