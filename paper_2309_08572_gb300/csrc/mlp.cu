// MLP surrogate on the GPU: forward, backward and Adam kernels (FP32), behind the C ABI.
//
// Not a method of the paper: a small fully connected network (tanh hidden layers, linear
// output) learns (energy per site, success probability) of noisy QAOA circuits from
// samples the MPDO engine produced, and its input gradient proposes angles that the
// engine then re-scores.
//   forward   z_l = a_{l-1} W_l + b_l, a_l = tanh(z_l) (hidden), a_L = z_L
//   loss      mean over batch and outputs of (a_L - t)^2
//   backward  dz_L = 2 (a_L - t) / (B n_out), dz_l = da_l (1 - a_l^2),
//             dW_l = a_{l-1}^T dz_l, db_l = column sums of dz_l, da_{l-1} = dz_l W_l^T
//   Adam      (Kingma & Ba) with bias correction.
// Weights are stored [fan_in][fan_out] row-major, one flat FP32 array W_0 b_0 W_1 b_1 ...
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "../../include/mpdo.h"
#include "common.cuh"
#include "tcgemm.h"

namespace mpdo {
void set_global_error(const char* msg);
}

namespace {

constexpr int SBM = 64, SBN = 64, SBK = 16, SNT = 256;

// C = op(A) op(B), A is M x K after op, B is K x N after op (row-major storage).
__global__ void __launch_bounds__(SNT) sgemm_kernel(int M, int N, int K, const float* __restrict__ A,
                                                    long sam, long sak, const float* __restrict__ B,
                                                    long sbk, long sbn, float* C, long ldc,
                                                    const float* __restrict__ bias) {
  __shared__ float As[SBK][SBM + 4];
  __shared__ float Bs[SBK][SBN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * SBM, n0 = blockIdx.x * SBN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += SBK) {
    for (int e = tid; e < SBM * SBK; e += SNT) {
      int mi, ki;
      if (sak == 1) { mi = e / SBK; ki = e % SBK; } else { ki = e / SBM; mi = e % SBM; }
      int gm = m0 + mi, gk = k0 + ki;
      As[ki][mi] = (gm < M && gk < K) ? A[gm * sam + gk * sak] : 0.f;
    }
    for (int e = tid; e < SBN * SBK; e += SNT) {
      int ni, ki;
      if (sbn == 1) { ki = e / SBN; ni = e % SBN; } else { ni = e / SBK; ki = e % SBK; }
      int gn = n0 + ni, gk = k0 + ki;
      Bs[ki][ni] = (gn < N && gk < K) ? B[gk * sbk + gn * sbn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      C[gm * ldc + gn] = acc[i][j] + (bias ? bias[gn] : 0.f);
    }
  }
}

__global__ void tanh_kernel(long n, float* z) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    z[e] = tanhf(z[e]);
}

// dz = 2 (y - t) / (B n_out); per-block partial sums of (y - t)^2 into part[]
__global__ void mse_grad_kernel(long n, float scale, const float* __restrict__ y,
                                const float* __restrict__ t, float* dz, double* part) {
  __shared__ double red[256];
  double s = 0;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    float d = y[e] - t[e];
    dz[e] = 2.f * d * scale;
    s += (double)d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// da <- da * (1 - a^2)
__global__ void tanh_back_kernel(long n, const float* __restrict__ a, float* da) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    float v = a[e];
    da[e] *= (1.f - v * v);
  }
}

// db[j] = sum_i dz[i][j]
__global__ void colsum_kernel(int rows, int cols, const float* __restrict__ dz, float* db) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int i = 0; i < rows; ++i) s += dz[(long)i * cols + j];
  db[j] = s;
}

__global__ void fill_rows_kernel(int rows, int cols, const float* __restrict__ v, float* out) {
  long n = (long)rows * cols;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    out[e] = v[e % cols];
}

__global__ void adam_kernel(long n, float lr, float b1, float b2, float eps, float c1, float c2,
                            const float* __restrict__ g, float* m, float* v, float* p) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    float gi = g[e];
    float mi = b1 * m[e] + (1.f - b1) * gi;
    float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

inline int nb(long n) {
  long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

struct mpdo_mlp_s {
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::vector<int> w;       // widths, size L+1
  int max_batch = 0;
  long n_params = 0;
  std::vector<long> woff, boff;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  std::vector<float*> acts;  // L+1 buffers, [max_batch][w_l]
  float *da = nullptr, *db2 = nullptr;  // two scratch [max_batch][max width]
  double* part = nullptr;
  double* hpart = nullptr;   // pinned
  int t = 0;
  int maxw = 0;
  std::string err;
  // BF16 tensor-core products (mpdo_mlp_set_precision): packed operands and the pipeline's
  // error flag; the parameters, gradients and Adam moments stay FP32
  int tc = 0;
  void *pa = nullptr, *pb = nullptr;
  int* tcerr = nullptr;
};

namespace {

int mlp_fail(mpdo_mlp m, int code, const std::string& msg) {
  if (m) m->err = msg;
  mpdo::set_global_error(msg.c_str());
  return code;
}

#define MK(expr)                                                                      \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) return mlp_fail(m, MPDO_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

__global__ void add_bias_kernel(int M, int N, float* C, long ldc, const float* __restrict__ bias) {
  const long total = (long)M * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x)
    C[(e / N) * ldc + e % N] += bias[e % N];
}

// C = op(A) op(B) (+ bias per column), A is M x K after op, B is K x N after op.  FP32 on the
// CUDA cores, or (m->tc) BF16 operands on the tensor cores with FP32 accumulation: op(A) and
// op(B)^T are packed K-major in BF16 and multiplied by the tcgen05 core.
cudaError_t sgemm(mpdo_mlp m, bool ta, bool tb, int M, int N, int K, const float* A, long lda,
                  const float* B, long ldb, float* C, long ldc, const float* bias) {
  cudaStream_t st = m->st;
  long sam = ta ? 1 : lda, sak = ta ? lda : 1;
  long sbk = tb ? 1 : ldb, sbn = tb ? ldb : 1;
  if (m->tc && M > 0 && N > 0 && K > 0) {
    const long ldk = (K + 7) / 8 * 8;   // 16-byte rows
    MPDO_CUDA_TRY(mpdo::tc_pack_real_bf16(st, M, K, A, sam, sak, m->pa, ldk));
    MPDO_CUDA_TRY(mpdo::tc_pack_real_bf16(st, N, K, B, sbn, sbk, m->pb, ldk));
    mpdo::TcEpilogue e;
    e.d = C;
    e.ldd = ldc;
    MPDO_CUDA_TRY(mpdo::tc_gemm_real(st, 2, M, N, K, m->pa, ldk, 0, m->pb, ldk, 0, 1, e,
                                     m->tcerr, 0));
    if (bias) {
      mpdo::count_launch();
      add_bias_kernel<<<nb((long)M * N), 256, 0, st>>>(M, N, C, ldc, bias);
    }
    return cudaGetLastError();
  }
  dim3 grid((N + SBN - 1) / SBN, (M + SBM - 1) / SBM);
  mpdo::count_launch();
  sgemm_kernel<<<grid, SNT, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias);
  return cudaGetLastError();
}

// forward pass into m->acts (acts[0] must hold x)
int run_forward(mpdo_mlp m, int batch) {
  const int L = (int)m->w.size() - 1;
  for (int l = 0; l < L; ++l) {
    MK(sgemm(m, false, false, batch, m->w[l + 1], m->w[l], m->acts[l], m->w[l],
             m->params + m->woff[l], m->w[l + 1], m->acts[l + 1], m->w[l + 1],
             m->params + m->boff[l]));
    if (l < L - 1) {
      long n = (long)batch * m->w[l + 1];
      mpdo::count_launch();
      tanh_kernel<<<nb(n), 256, 0, m->st>>>(n, m->acts[l + 1]);
      MK(cudaGetLastError());
    }
  }
  return MPDO_OK;
}

// backward from d(output) in m->da; fills m->grads if want_params; leaves d(input) in m->da
int run_backward(mpdo_mlp m, int batch, bool want_params) {
  const int L = (int)m->w.size() - 1;
  float* cur = m->da;
  float* nxt = m->db2;
  for (int l = L - 1; l >= 0; --l) {
    const int fi = m->w[l], fo = m->w[l + 1];
    if (l < L - 1) {
      long n = (long)batch * fo;
      mpdo::count_launch();
      tanh_back_kernel<<<nb(n), 256, 0, m->st>>>(n, m->acts[l + 1], cur);
      MK(cudaGetLastError());
    }
    if (want_params) {
      // dW = a_{l-1}^T dz  (fi x fo), db = colsum(dz)
      MK(sgemm(m, true, false, fi, fo, batch, m->acts[l], fi, cur, fo, m->grads + m->woff[l],
               fo, nullptr));
      mpdo::count_launch();
      colsum_kernel<<<(fo + 127) / 128, 128, 0, m->st>>>(batch, fo, cur, m->grads + m->boff[l]);
      MK(cudaGetLastError());
    }
    // da_{l-1} = dz W^T  (batch x fi)
    MK(sgemm(m, false, true, batch, fi, fo, cur, fo, m->params + m->woff[l], fo, nxt, fi,
             nullptr));
    std::swap(cur, nxt);
  }
  if (cur != m->da) MK(cudaMemcpyAsync(m->da, cur, sizeof(float) * (size_t)batch * m->w[0],
                                       cudaMemcpyDeviceToDevice, m->st));
  return MPDO_OK;
}

}  // namespace

extern "C" {

int mpdo_mlp_create(int n_layers, const int* widths, int max_batch, void* stream, mpdo_mlp* out) {
  if (n_layers < 1 || n_layers > 16 || !widths || max_batch < 1 || !out)
    return mlp_fail(nullptr, MPDO_ERR_ARG, "mlp: bad create arguments");
  for (int l = 0; l <= n_layers; ++l)
    if (widths[l] < 1 || widths[l] > 4096) return mlp_fail(nullptr, MPDO_ERR_ARG, "mlp: width out of 1..4096");
  mpdo_mlp m = new (std::nothrow) mpdo_mlp_s();
  if (!m) return mlp_fail(nullptr, MPDO_ERR_OOM, "mlp: host allocation");
  m->w.assign(widths, widths + n_layers + 1);
  m->max_batch = max_batch;
  long off = 0;
  for (int l = 0; l < n_layers; ++l) {
    m->woff.push_back(off);
    off += (long)m->w[l] * m->w[l + 1];
    m->boff.push_back(off);
    off += m->w[l + 1];
  }
  m->n_params = off;
  for (int x : m->w) m->maxw = std::max(m->maxw, x);
  if (stream) {
    m->st = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete m;
      return mlp_fail(nullptr, MPDO_ERR_CUDA, "mlp: stream creation");
    }
    m->own_stream = true;
  }
  bool ok = cudaMalloc(&m->params, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&m->grads, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&m->m, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&m->v, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&m->da, sizeof(float) * (size_t)max_batch * m->maxw) == cudaSuccess &&
            cudaMalloc(&m->db2, sizeof(float) * (size_t)max_batch * m->maxw) == cudaSuccess &&
            cudaMalloc(&m->part, sizeof(double) * 4096) == cudaSuccess &&
            cudaMallocHost(&m->hpart, sizeof(double) * 4096) == cudaSuccess;
  for (int l = 0; ok && l <= n_layers; ++l) {
    float* p = nullptr;
    ok = cudaMalloc(&p, sizeof(float) * (size_t)max_batch * m->w[l]) == cudaSuccess;
    m->acts.push_back(p);
  }
  if (!ok) {
    cudaGetLastError();
    mpdo_mlp_destroy(m);
    return mlp_fail(nullptr, MPDO_ERR_OOM, "mlp: device allocation");
  }
  cudaMemsetAsync(m->params, 0, sizeof(float) * off, m->st);
  cudaMemsetAsync(m->m, 0, sizeof(float) * off, m->st);
  cudaMemsetAsync(m->v, 0, sizeof(float) * off, m->st);
  cudaStreamSynchronize(m->st);
  *out = m;
  return MPDO_OK;
}

long long mpdo_mlp_n_params(mpdo_mlp m) { return m ? m->n_params : -1; }

int mpdo_mlp_set_params(mpdo_mlp m, const float* host) {
  if (!m || !host) return mlp_fail(m, MPDO_ERR_ARG, "mlp: null argument");
  for (long i = 0; i < m->n_params; ++i)
    if (!std::isfinite(host[i])) return mlp_fail(m, MPDO_ERR_NUMERIC, "mlp: non-finite parameter");
  MK(cudaMemcpyAsync(m->params, host, sizeof(float) * m->n_params, cudaMemcpyHostToDevice, m->st));
  MK(cudaMemsetAsync(m->m, 0, sizeof(float) * m->n_params, m->st));
  MK(cudaMemsetAsync(m->v, 0, sizeof(float) * m->n_params, m->st));
  MK(cudaStreamSynchronize(m->st));
  m->t = 0;
  return MPDO_OK;
}

int mpdo_mlp_get_params(mpdo_mlp m, float* host) {
  if (!m || !host) return mlp_fail(m, MPDO_ERR_ARG, "mlp: null argument");
  MK(cudaMemcpyAsync(host, m->params, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, m->st));
  MK(cudaStreamSynchronize(m->st));
  return MPDO_OK;
}

int mpdo_mlp_forward(mpdo_mlp m, int batch, const float* x, float* y) {
  if (!m || !x || !y || batch < 1 || batch > m->max_batch) return mlp_fail(m, MPDO_ERR_ARG, "mlp: bad forward arguments");
  MK(cudaMemcpyAsync(m->acts[0], x, sizeof(float) * (size_t)batch * m->w[0], cudaMemcpyDeviceToDevice, m->st));
  int rc = run_forward(m, batch);
  if (rc) return rc;
  const int L = (int)m->w.size() - 1;
  MK(cudaMemcpyAsync(y, m->acts[L], sizeof(float) * (size_t)batch * m->w[L], cudaMemcpyDeviceToDevice, m->st));
  return MPDO_OK;
}

int mpdo_mlp_loss_grad(mpdo_mlp m, int batch, const float* x, const float* t, float* loss,
                       float* grad_host) {
  if (!m || !x || !t || batch < 1 || batch > m->max_batch) return mlp_fail(m, MPDO_ERR_ARG, "mlp: bad loss_grad arguments");
  MK(cudaMemcpyAsync(m->acts[0], x, sizeof(float) * (size_t)batch * m->w[0], cudaMemcpyDeviceToDevice, m->st));
  int rc = run_forward(m, batch);
  if (rc) return rc;
  const int L = (int)m->w.size() - 1;
  const long n = (long)batch * m->w[L];
  const int blocks = nb(n);
  mpdo::count_launch();
  mse_grad_kernel<<<blocks, 256, 0, m->st>>>(n, 1.f / (float)n, m->acts[L], t, m->da, m->part);
  MK(cudaGetLastError());
  rc = run_backward(m, batch, true);
  if (rc) return rc;
  MK(cudaMemcpyAsync(m->hpart, m->part, sizeof(double) * blocks, cudaMemcpyDeviceToHost, m->st));
  if (grad_host) MK(cudaMemcpyAsync(grad_host, m->grads, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, m->st));
  if (m->tc) MK(cudaMemcpyAsync(m->hpart + 4095, m->tcerr, sizeof(int), cudaMemcpyDeviceToHost, m->st));
  MK(cudaStreamSynchronize(m->st));
  if (m->tc && *reinterpret_cast<int*>(m->hpart + 4095))
    return mlp_fail(m, MPDO_ERR_TIMEOUT, "mlp: a tensor-core pipeline wait gave up");
  double s = 0;
  for (int b = 0; b < blocks; ++b) s += m->hpart[b];
  if (loss) *loss = (float)(s / (double)n);
  return MPDO_OK;
}

int mpdo_mlp_adam_step(mpdo_mlp m, float lr) {
  if (!m || !(lr > 0)) return mlp_fail(m, MPDO_ERR_ARG, "mlp: bad learning rate");
  m->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)m->t), c2 = 1.f - powf(b2, (float)m->t);
  mpdo::count_launch();
  adam_kernel<<<nb(m->n_params), 256, 0, m->st>>>(m->n_params, lr, b1, b2, 1e-8f, c1, c2, m->grads,
                                                  m->m, m->v, m->params);
  MK(cudaGetLastError());
  return MPDO_OK;
}

int mpdo_mlp_input_grad(mpdo_mlp m, int batch, const float* x, const float* wout_host, float* gx) {
  if (!m || !x || !wout_host || !gx || batch < 1 || batch > m->max_batch)
    return mlp_fail(m, MPDO_ERR_ARG, "mlp: bad input_grad arguments");
  MK(cudaMemcpyAsync(m->acts[0], x, sizeof(float) * (size_t)batch * m->w[0], cudaMemcpyDeviceToDevice, m->st));
  int rc = run_forward(m, batch);
  if (rc) return rc;
  const int L = (int)m->w.size() - 1;
  // d(output) = wout broadcast over rows
  MK(cudaMemcpyAsync(m->db2, wout_host, sizeof(float) * m->w[L], cudaMemcpyHostToDevice, m->st));
  mpdo::count_launch();
  fill_rows_kernel<<<nb((long)batch * m->w[L]), 256, 0, m->st>>>(batch, m->w[L], m->db2, m->da);
  MK(cudaGetLastError());
  rc = run_backward(m, batch, false);
  if (rc) return rc;
  MK(cudaMemcpyAsync(gx, m->da, sizeof(float) * (size_t)batch * m->w[0], cudaMemcpyDeviceToDevice, m->st));
  MK(cudaStreamSynchronize(m->st));
  return MPDO_OK;
}

int mpdo_mlp_set_precision(mpdo_mlp m, int mode) {
  if (!m || (mode != 0 && mode != 1)) return mlp_fail(m, MPDO_ERR_ARG, "mlp: precision mode must be 0 or 1");
  MK(cudaStreamSynchronize(m->st));
  if (mode == 1 && !m->pa) {
    const long r = std::max(m->max_batch, m->maxw), ldk = (r + 7) / 8 * 8;
    const size_t bytes = (size_t)r * ldk * 2;
    if (cudaMalloc(&m->pa, bytes) != cudaSuccess || cudaMalloc(&m->pb, bytes) != cudaSuccess ||
        cudaMalloc(&m->tcerr, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return mlp_fail(m, MPDO_ERR_OOM, "mlp: tensor-core operand buffers");
    }
    MK(cudaMemsetAsync(m->tcerr, 0, sizeof(int), m->st));
  }
  m->tc = mode;
  return MPDO_OK;
}

int mpdo_mlp_destroy(mpdo_mlp m) {
  if (!m) return MPDO_OK;
  if (m->st) cudaStreamSynchronize(m->st);
  if (m->pa) cudaFree(m->pa);
  if (m->pb) cudaFree(m->pb);
  if (m->tcerr) cudaFree(m->tcerr);
  for (float* p : m->acts) if (p) cudaFree(p);
  if (m->params) cudaFree(m->params);
  if (m->grads) cudaFree(m->grads);
  if (m->m) cudaFree(m->m);
  if (m->v) cudaFree(m->v);
  if (m->da) cudaFree(m->da);
  if (m->db2) cudaFree(m->db2);
  if (m->part) cudaFree(m->part);
  if (m->hpart) cudaFreeHost(m->hpart);
  if (m->own_stream) cudaStreamDestroy(m->st);
  delete m;
  return MPDO_OK;
}

}  // extern "C"
