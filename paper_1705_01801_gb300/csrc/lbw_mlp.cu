// lbw_mlp.cu -- a small multilayer perceptron, trained and evaluated on the device, used as a
// surrogate from ensemble geometry parameters to the lowest mode frequencies the batched
// lattice-Boltzmann runs measure (the paper has no counterpart; the LBM stays the reference).
//
// Network: depth weight layers, in -> hidden -> ... -> hidden -> out, tanh after every layer
// but the last (linear).  Loss: mean over samples and outputs of (y - t)^2.  Parameters are one
// FP32 vector: for each layer W (out x in, row-major) then b (out).  Training: Adam on
// minibatches whose order comes from the caller.  Inference also exists with weights stored
// in BF16 (FP32 accumulation).  All arithmetic runs in the kernels below: a tiled FP32 GEMM
// (C = op(A) op(B) with transposes for the backward pass), bias / activation / loss kernels,
// a column-sum reduction for bias gradients and the Adam update.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "lbw_internal.h"

namespace lbw {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;  // GEMM tile; 256 threads, 4 x 4 outputs each

// C[m x n] = op(A) op(B) (+ bias[n]); op(A) is m x k (A stored k x m when ta), op(B) is k x n
// (B stored n x k when tb).  Leading dimensions are the stored row lengths.
template <typename WB>
__global__ void __launch_bounds__(256) gemm_kernel(const float* __restrict__ A, int lda, bool ta,
                                                   const WB* __restrict__ B, int ldb, bool tb,
                                                   float* __restrict__ C, int ldc, int m, int n, int k,
                                                   const float* __restrict__ bias, bool accumulate) {
  __shared__ float As[TK][TM + 1];
  __shared__ float Bs[TK][TN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < k; k0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      const int r = e / TK, c = e % TK;  // tile row (m), tile col (k)
      const int gm = row0 + r, gk = k0 + c;
      float v = 0.f;
      if (gm < m && gk < k) v = ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[c][r] = v;
    }
    for (int e = threadIdx.x; e < TN * TK; e += 256) {
      const int r = e / TK, c = e % TK;  // tile col (n), k index
      const int gn = col0 + r, gk = k0 + c;
      float v = 0.f;
      if (gn < n && gk < k) v = (float)(tb ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn]);
      Bs[c][r] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = row0 + ty * 4 + i, gn = col0 + tx * 4 + j;
      if (gm < m && gn < n) {
        float v = acc[i][j] + (bias ? bias[gn] : 0.f);
        if (accumulate) v += C[(size_t)gm * ldc + gn];
        C[(size_t)gm * ldc + gn] = v;
      }
    }
}

__global__ void bias_act_kernel(float* __restrict__ Y, const float* __restrict__ b, int m, int n, bool act) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * n; e += gridDim.x * blockDim.x) {
    float v = Y[e] + b[e % n];
    Y[e] = act ? tanhf(v) : v;
  }
}

// dY = 2 (y - t) / (m n); loss partial sums per block
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                           int count, float* __restrict__ loss) {
  __shared__ float red[256];
  float s = 0.f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    const float d = y[e] - t[e];
    dy[e] = 2.f * d / (float)count;
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / (float)count);
}

// dZ = dY (1 - y^2) through tanh, in place on dY
__global__ void tanh_back_kernel(float* __restrict__ d, const float* __restrict__ y, int count) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
    d[e] *= 1.f - y[e] * y[e];
}

// db[j] = sum_i dZ[i, j]
__global__ void colsum_kernel(const float* __restrict__ d, int m, int n, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float s = 0.f;
  for (int i = 0; i < m; ++i) s += d[(size_t)i * n + j];
  out[j] = s;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, int count, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float a = b1 * m1[e] + (1.f - b1) * gi;
    const float v = b2 * m2[e] + (1.f - b2) * gi * gi;
    m1[e] = a;
    m2[e] = v;
    p[e] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
  }
}

__global__ void gather_rows_kernel(const float* __restrict__ src, const int* __restrict__ idx, int rows,
                                   int cols, float* __restrict__ dst) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols; e += gridDim.x * blockDim.x)
    dst[e] = src[(size_t)idx[e / cols] * cols + e % cols];
}

__global__ void to_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ q, int count) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
    q[e] = __float2bfloat16_rn(p[e]);
}

}  // namespace
}  // namespace lbw

using namespace lbw;

struct lbw_mlp {
  int in = 0, hidden = 0, depth = 0, out = 0;
  std::vector<int> dims;         // depth + 1 layer widths
  std::vector<size_t> woff, boff;  // parameter offsets of each layer
  size_t nparam = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
  __nv_bfloat16* pb = nullptr;   // BF16 copy for inference
  bool pb_valid = false;
  long long adam_t = 0;
  // work buffers for up to cap rows
  int cap = 0;
  std::vector<float*> act;       // activations per layer (depth + 1), cap x width
  float *delta = nullptr, *delta2 = nullptr, *target = nullptr, *loss = nullptr;
  int* idx = nullptr;
  float *data_x = nullptr, *data_t = nullptr;
  int data_n = 0;
};

namespace {

void free_work(lbw_mlp* q) {
  for (float* a : q->act)
    if (a) cudaFreeAsync(a, q->stream);
  q->act.clear();
  float** bufs[] = {&q->delta, &q->delta2, &q->target, &q->loss};
  for (float** b : bufs)
    if (*b) { cudaFreeAsync(*b, q->stream); *b = nullptr; }
  if (q->idx) { cudaFreeAsync(q->idx, q->stream); q->idx = nullptr; }
  q->cap = 0;
}

lbw_status ensure_work(lbw_mlp* q, int rows) {
  if (rows <= q->cap) return LBW_OK;
  free_work(q);
  int maxw = 0;
  for (int w : q->dims) maxw = std::max(maxw, w);
  q->act.assign(q->dims.size(), nullptr);
  for (size_t l = 0; l < q->dims.size(); ++l)
    LBW_CUDA(cudaMallocAsync((void**)&q->act[l], sizeof(float) * rows * q->dims[l], q->stream));
  LBW_CUDA(cudaMallocAsync((void**)&q->delta, sizeof(float) * rows * maxw, q->stream));
  LBW_CUDA(cudaMallocAsync((void**)&q->delta2, sizeof(float) * rows * maxw, q->stream));
  LBW_CUDA(cudaMallocAsync((void**)&q->target, sizeof(float) * rows * q->out, q->stream));
  LBW_CUDA(cudaMallocAsync((void**)&q->loss, sizeof(float), q->stream));
  LBW_CUDA(cudaMallocAsync((void**)&q->idx, sizeof(int) * rows, q->stream));
  q->cap = rows;
  return LBW_OK;
}

dim3 gemm_grid(int m, int n) { return dim3((n + TN - 1) / TN, (m + TM - 1) / TM); }

// forward through all layers for act[0] (rows x in) already on the device
template <typename WB>
void forward(lbw_mlp* q, int rows, const WB* params) {
  for (int l = 0; l < q->depth; ++l) {
    const int in = q->dims[l], out = q->dims[l + 1];
    gemm_kernel<WB><<<gemm_grid(rows, out), 256, 0, q->stream>>>(q->act[l], in, false, params + q->woff[l], in,
                                                                  true, q->act[l + 1], out, rows, out, in,
                                                                  nullptr, false);
    bias_act_kernel<<<152 * 4, 256, 0, q->stream>>>(q->act[l + 1], q->p + q->boff[l], rows, out, l + 1 < q->depth);
  }
}

// loss and parameter gradient (into q->g) for act[0] and target on the device
void backward(lbw_mlp* q, int rows) {
  const int last = q->depth;
  const int cnt = rows * q->out;
  cudaMemsetAsync(q->loss, 0, sizeof(float), q->stream);
  mse_kernel<<<152, 256, 0, q->stream>>>(q->act[last], q->target, q->delta, cnt, q->loss);
  for (int l = q->depth - 1; l >= 0; --l) {
    const int in = q->dims[l], out = q->dims[l + 1];
    if (l + 1 < q->depth) tanh_back_kernel<<<152 * 4, 256, 0, q->stream>>>(q->delta, q->act[l + 1], rows * out);
    // dW = dZ^T X  (out x in)
    gemm_kernel<float><<<gemm_grid(out, in), 256, 0, q->stream>>>(q->delta, out, true, q->act[l], in, false,
                                                                   q->g + q->woff[l], in, out, in, rows,
                                                                   nullptr, false);
    colsum_kernel<<<(out + 255) / 256, 256, 0, q->stream>>>(q->delta, rows, out, q->g + q->boff[l]);
    if (l > 0) {
      // dX = dZ W  (rows x in)
      gemm_kernel<float><<<gemm_grid(rows, in), 256, 0, q->stream>>>(q->delta, out, false, q->p + q->woff[l], in,
                                                                      false, q->delta2, in, rows, in, out,
                                                                      nullptr, false);
      std::swap(q->delta, q->delta2);
    }
  }
}

unsigned long long splitmix(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

}  // namespace

extern "C" {

lbw_status lbw_mlp_create(int32_t in_dim, int32_t hidden, int32_t depth, int32_t out_dim, uint64_t seed,
                          void* stream, lbw_mlp** out) {
  if (!out) return fail(LBW_EINVAL, "out is NULL");
  *out = nullptr;
  if (in_dim < 1 || in_dim > 4096 || hidden < 1 || hidden > 4096 || out_dim < 1 || out_dim > 4096 ||
      depth < 1 || depth > 16)
    return fail(LBW_EINVAL, "dimensions out of range (1..4096, depth 1..16)");
  lbw_mlp* q = new (std::nothrow) lbw_mlp();
  if (!q) return fail(LBW_ENOMEM, "host allocation failed");
  q->in = in_dim; q->hidden = hidden; q->depth = depth; q->out = out_dim;
  q->dims.push_back(in_dim);
  for (int l = 0; l + 1 < depth; ++l) q->dims.push_back(hidden);
  q->dims.push_back(out_dim);
  size_t off = 0;
  for (int l = 0; l < depth; ++l) {
    q->woff.push_back(off);
    off += (size_t)q->dims[l + 1] * q->dims[l];
    q->boff.push_back(off);
    off += q->dims[l + 1];
  }
  q->nparam = off;
  q->stream = reinterpret_cast<cudaStream_t>(stream);
  if (!q->stream) {
    if (cudaStreamCreate(&q->stream) != cudaSuccess) {
      delete q;
      return fail(LBW_ECUDA, "cudaStreamCreate failed");
    }
    q->own_stream = true;
  }
  // uniform(-s, s) with s = sqrt(6 / (fan_in + fan_out)) from a counter-based generator
  std::vector<float> h(q->nparam, 0.f);
  for (int l = 0; l < depth; ++l) {
    const double s = std::sqrt(6.0 / (q->dims[l] + q->dims[l + 1]));
    for (size_t e = 0; e < (size_t)q->dims[l + 1] * q->dims[l]; ++e) {
      const double u = (splitmix(seed ^ (q->woff[l] + e) * 0x2545F4914F6CDD1DULL) >> 11) * (1.0 / 9007199254740992.0);
      h[q->woff[l] + e] = (float)((2.0 * u - 1.0) * s);
    }
  }
  cudaError_t e = cudaMallocAsync((void**)&q->p, sizeof(float) * q->nparam, q->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&q->g, sizeof(float) * q->nparam, q->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&q->m1, sizeof(float) * q->nparam, q->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&q->m2, sizeof(float) * q->nparam, q->stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&q->pb, sizeof(__nv_bfloat16) * q->nparam, q->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(q->p, h.data(), sizeof(float) * q->nparam, cudaMemcpyHostToDevice, q->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(q->m1, 0, sizeof(float) * q->nparam, q->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(q->m2, 0, sizeof(float) * q->nparam, q->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
  if (e != cudaSuccess) {
    lbw_mlp_destroy(q);
    return cuda_fail(e, "mlp create");
  }
  *out = q;
  return LBW_OK;
}

void lbw_mlp_destroy(lbw_mlp* q) {
  if (!q) return;
  free_work(q);
  float* bufs[] = {q->p, q->g, q->m1, q->m2, q->data_x, q->data_t};
  for (float* b : bufs)
    if (b) cudaFreeAsync(b, q->stream);
  if (q->pb) cudaFreeAsync(q->pb, q->stream);
  cudaStreamSynchronize(q->stream);
  if (q->own_stream) cudaStreamDestroy(q->stream);
  delete q;
}

lbw_status lbw_mlp_param_count(lbw_mlp* q, int64_t* n) {
  if (!q || !n) return fail(LBW_EINVAL, "NULL argument");
  *n = (int64_t)q->nparam;
  return LBW_OK;
}

lbw_status lbw_mlp_get_params(lbw_mlp* q, float* host_params) {
  if (!q || !host_params) return fail(LBW_EINVAL, "NULL argument");
  LBW_CUDA(cudaMemcpyAsync(host_params, q->p, sizeof(float) * q->nparam, cudaMemcpyDeviceToHost, q->stream));
  LBW_CUDA(cudaStreamSynchronize(q->stream));
  return LBW_OK;
}

lbw_status lbw_mlp_set_params(lbw_mlp* q, const float* host_params) {
  if (!q || !host_params) return fail(LBW_EINVAL, "NULL argument");
  LBW_CUDA(cudaMemcpyAsync(q->p, host_params, sizeof(float) * q->nparam, cudaMemcpyHostToDevice, q->stream));
  LBW_CUDA(cudaMemsetAsync(q->m1, 0, sizeof(float) * q->nparam, q->stream));
  LBW_CUDA(cudaMemsetAsync(q->m2, 0, sizeof(float) * q->nparam, q->stream));
  LBW_CUDA(cudaStreamSynchronize(q->stream));
  q->adam_t = 0;
  q->pb_valid = false;
  return LBW_OK;
}

lbw_status lbw_mlp_forward(lbw_mlp* q, const float* host_x, int32_t n, float* host_y) {
  if (!q || !host_x || !host_y || n < 1) return fail(LBW_EINVAL, "bad argument");
  lbw_status st = ensure_work(q, n);
  if (st != LBW_OK) return st;
  LBW_CUDA(cudaMemcpyAsync(q->act[0], host_x, sizeof(float) * n * q->in, cudaMemcpyHostToDevice, q->stream));
  forward<float>(q, n, q->p);
  LBW_CUDA(cudaGetLastError());
  LBW_CUDA(cudaMemcpyAsync(host_y, q->act[q->depth], sizeof(float) * n * q->out, cudaMemcpyDeviceToHost, q->stream));
  LBW_CUDA(cudaStreamSynchronize(q->stream));
  return LBW_OK;
}

lbw_status lbw_mlp_predict_bf16(lbw_mlp* q, const float* host_x, int32_t n, float* host_y) {
  if (!q || !host_x || !host_y || n < 1) return fail(LBW_EINVAL, "bad argument");
  lbw_status st = ensure_work(q, n);
  if (st != LBW_OK) return st;
  if (!q->pb_valid) {
    to_bf16_kernel<<<152 * 4, 256, 0, q->stream>>>(q->p, q->pb, (int)q->nparam);
    q->pb_valid = true;
  }
  LBW_CUDA(cudaMemcpyAsync(q->act[0], host_x, sizeof(float) * n * q->in, cudaMemcpyHostToDevice, q->stream));
  forward<__nv_bfloat16>(q, n, q->pb);
  LBW_CUDA(cudaGetLastError());
  LBW_CUDA(cudaMemcpyAsync(host_y, q->act[q->depth], sizeof(float) * n * q->out, cudaMemcpyDeviceToHost, q->stream));
  LBW_CUDA(cudaStreamSynchronize(q->stream));
  return LBW_OK;
}

lbw_status lbw_mlp_grad(lbw_mlp* q, const float* host_x, const float* host_t, int32_t n, float* host_grad,
                        float* host_loss) {
  if (!q || !host_x || !host_t || n < 1) return fail(LBW_EINVAL, "bad argument");
  lbw_status st = ensure_work(q, n);
  if (st != LBW_OK) return st;
  LBW_CUDA(cudaMemcpyAsync(q->act[0], host_x, sizeof(float) * n * q->in, cudaMemcpyHostToDevice, q->stream));
  LBW_CUDA(cudaMemcpyAsync(q->target, host_t, sizeof(float) * n * q->out, cudaMemcpyHostToDevice, q->stream));
  forward<float>(q, n, q->p);
  backward(q, n);
  LBW_CUDA(cudaGetLastError());
  if (host_grad)
    LBW_CUDA(cudaMemcpyAsync(host_grad, q->g, sizeof(float) * q->nparam, cudaMemcpyDeviceToHost, q->stream));
  if (host_loss) LBW_CUDA(cudaMemcpyAsync(host_loss, q->loss, sizeof(float), cudaMemcpyDeviceToHost, q->stream));
  LBW_CUDA(cudaStreamSynchronize(q->stream));
  return LBW_OK;
}

lbw_status lbw_mlp_adam_step(lbw_mlp* q, const float* host_grad, float lr) {
  if (!q || !host_grad) return fail(LBW_EINVAL, "NULL argument");
  LBW_CUDA(cudaMemcpyAsync(q->g, host_grad, sizeof(float) * q->nparam, cudaMemcpyHostToDevice, q->stream));
  ++q->adam_t;
  const float b1 = 0.9f, b2 = 0.999f;
  adam_kernel<<<152 * 4, 256, 0, q->stream>>>(q->p, q->g, q->m1, q->m2, (int)q->nparam, lr, b1, b2, 1e-8f,
                                               (float)(1.0 - std::pow(0.9, (double)q->adam_t)),
                                               (float)(1.0 - std::pow(0.999, (double)q->adam_t)));
  LBW_CUDA(cudaGetLastError());
  LBW_CUDA(cudaStreamSynchronize(q->stream));
  q->pb_valid = false;
  return LBW_OK;
}

lbw_status lbw_mlp_train(lbw_mlp* q, const float* host_x, const float* host_t, int32_t n,
                         const int32_t* host_order, int32_t n_steps, int32_t batch, float lr, float* host_loss) {
  if (!q || !host_x || !host_t || !host_order || n < 1 || n_steps < 0 || batch < 1 || batch > n)
    return fail(LBW_EINVAL, "bad argument");
  for (long long e = 0; e < (long long)n_steps * batch; ++e)
    if (host_order[e] < 0 || host_order[e] >= n) return fail(LBW_EINVAL, "host_order holds an index outside [0, n)");
  lbw_status st = ensure_work(q, batch);
  if (st != LBW_OK) return st;
  if (q->data_n != n) {
    if (q->data_x) cudaFreeAsync(q->data_x, q->stream);
    if (q->data_t) cudaFreeAsync(q->data_t, q->stream);
    LBW_CUDA(cudaMallocAsync((void**)&q->data_x, sizeof(float) * n * q->in, q->stream));
    LBW_CUDA(cudaMallocAsync((void**)&q->data_t, sizeof(float) * n * q->out, q->stream));
    q->data_n = n;
  }
  LBW_CUDA(cudaMemcpyAsync(q->data_x, host_x, sizeof(float) * n * q->in, cudaMemcpyHostToDevice, q->stream));
  LBW_CUDA(cudaMemcpyAsync(q->data_t, host_t, sizeof(float) * n * q->out, cudaMemcpyHostToDevice, q->stream));
  int* d_order = nullptr;
  LBW_CUDA(cudaMallocAsync((void**)&d_order, sizeof(int) * (size_t)n_steps * batch, q->stream));
  LBW_CUDA(cudaMemcpyAsync(d_order, host_order, sizeof(int) * (size_t)n_steps * batch, cudaMemcpyHostToDevice,
                           q->stream));
  float* d_curve = nullptr;
  LBW_CUDA(cudaMallocAsync((void**)&d_curve, sizeof(float) * std::max(1, n_steps), q->stream));
  const float b1 = 0.9f, b2 = 0.999f;
  for (int s = 0; s < n_steps; ++s) {
    gather_rows_kernel<<<64, 256, 0, q->stream>>>(q->data_x, d_order + (size_t)s * batch, batch, q->in, q->act[0]);
    gather_rows_kernel<<<64, 256, 0, q->stream>>>(q->data_t, d_order + (size_t)s * batch, batch, q->out, q->target);
    forward<float>(q, batch, q->p);
    backward(q, batch);
    cudaMemcpyAsync(d_curve + s, q->loss, sizeof(float), cudaMemcpyDeviceToDevice, q->stream);
    ++q->adam_t;
    adam_kernel<<<152 * 4, 256, 0, q->stream>>>(q->p, q->g, q->m1, q->m2, (int)q->nparam, lr, b1, b2, 1e-8f,
                                                 (float)(1.0 - std::pow(0.9, (double)q->adam_t)),
                                                 (float)(1.0 - std::pow(0.999, (double)q->adam_t)));
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && host_loss && n_steps > 0)
    e = cudaMemcpyAsync(host_loss, d_curve, sizeof(float) * n_steps, cudaMemcpyDeviceToHost, q->stream);
  cudaFreeAsync(d_order, q->stream);
  cudaFreeAsync(d_curve, q->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mlp train");
  q->pb_valid = false;
  return LBW_OK;
}

}  // extern "C"
