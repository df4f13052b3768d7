// Host side of the screening network (swcs_mlp_* in include/swcs.h).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/swcs.h"
#include "swcs_kernels.h"

using namespace swcs;

struct swcs_mlp {
  cudaStream_t st = nullptr;
  std::string err;
  MlpParams p{};
  float* grad = nullptr;
  double* loss = nullptr;
  int step = 0;
  // activations and scratch for up to cap rows
  int64_t cap = 0;
  __nv_bfloat16 *H1 = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
  __nv_bfloat16 *dZ2t = nullptr, *H1t = nullptr, *dZ1t = nullptr, *Xt = nullptr;
  float *y = nullptr, *dy = nullptr, *dH1 = nullptr;
  int* err_dev = nullptr;
  int64_t launches = 0;
  bool pipeline = true;  // option "gemm_pipeline"
};

namespace {

int mfail(swcs_mlp* m, int code, const std::string& msg) {
  if (m) m->err = msg;
  return code;
}

#define MCK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return mfail(m, SWCS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc((void**)p, n * sizeof(T));
}

void free_scratch(swcs_mlp* m) {
  void* bufs[] = {m->H1, m->H2, m->dZ2, m->dZ1, m->dZ2t, m->H1t, m->dZ1t, m->Xt, m->y, m->dy, m->dH1};
  for (void* b : bufs)
    if (b) cudaFree(b);
  m->H1 = m->H2 = m->dZ2 = m->dZ1 = m->dZ2t = m->H1t = m->dZ1t = m->Xt = nullptr;
  m->y = m->dy = m->dH1 = nullptr;
  m->cap = 0;
}

int ensure_rows(swcs_mlp* m, int64_t rows) {
  if (rows <= m->cap) return SWCS_OK;
  free_scratch(m);
  const int64_t r = ((rows + 127) / 128) * 128;
  const size_t W = (size_t)m->p.width, D = (size_t)m->p.d_in;
  if (dalloc(&m->H1, r * W) || dalloc(&m->H2, r * W) || dalloc(&m->dZ2, r * W) || dalloc(&m->dZ1, r * W) ||
      dalloc(&m->dZ2t, r * W) || dalloc(&m->H1t, r * W) || dalloc(&m->dZ1t, r * W) || dalloc(&m->Xt, r * D) ||
      dalloc(&m->y, r) || dalloc(&m->dy, r) || dalloc(&m->dH1, r * W)) {
    cudaGetLastError();
    free_scratch(m);
    return mfail(m, SWCS_ERR_OOM, "mlp: activation buffers");
  }
  m->cap = r;
  return SWCS_OK;
}

GemmArgs gemm(swcs_mlp* m, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
              int mode) {
  GemmArgs g{};
  g.A = A;
  g.B = B;
  g.lda = lda;
  g.ldb = ldb;
  g.M = M;
  g.N = N;
  g.K = K;
  g.mode = mode;
  g.err = m->err_dev;
  return g;
}

bool k_major_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows);

// C = A B^T through the pipelined kernel when both operands have tensor maps (K contiguous, 16-byte aligned),
// else through the staged one.  may_split: the FP32 output holds zeros, so K may be split over CTAs.
int run_gemm(swcs_mlp* m, const GemmArgs& g, bool may_split) {
  CUtensorMap ta, tb;
  if (m->pipeline && g.lda == g.K && g.ldb == g.K && k_major_map(&ta, g.A, (uint64_t)g.K, (uint64_t)g.M, 128) &&
      k_major_map(&tb, g.B, (uint64_t)g.K, (uint64_t)g.N, (uint32_t)g.N)) {
    int splits = 1;
    if (may_split && g.mode == kGemmF32) {
      int dev = 0, nsm = 0;
      MCK(cudaGetDevice(&dev));
      MCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      const int tiles = (g.M + 127) / 128, nch = g.K / mlp_gemm_tma_kc(g.K);
      splits = std::max(1, std::min(nch / 4, (2 * nsm) / tiles));  // at least four K-chunks per CTA
    }
    MCK(launch_mlp_gemm_tma(ta, tb, g, splits, m->st));
  } else {
    MCK(launch_mlp_gemm(g, m->st));
  }
  return SWCS_OK;
}

// forward into m->H1, m->H2, y
int forward(swcs_mlp* m, const __nv_bfloat16* x, int64_t n, float* y) {
  const int W = m->p.width, D = m->p.d_in;
  GemmArgs g1 = gemm(m, x, D, m->p.W1b, D, (int)n, W, D, kGemmReluBf16);
  g1.bias = m->p.master + m->p.off_b1;
  g1.out_bf16 = m->H1;
  g1.ldo = W;
  int r;
  if ((r = run_gemm(m, g1, false))) return r;
  GemmArgs g2 = gemm(m, m->H1, W, m->p.W2b, W, (int)n, W, W, kGemmReluBf16Dot);
  g2.bias = m->p.master + m->p.off_b2;
  g2.out_bf16 = m->H2;
  g2.ldo = W;
  g2.w3 = m->p.w3b;
  // b3 is read on the device side through the bias of a 1-column add: kept on host copy
  g2.b3 = 0.f;
  g2.y = y;
  if ((r = run_gemm(m, g2, false))) return r;
  m->launches += 2;
  return SWCS_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// Row-major BF16 [rows x inner] with boxes of 8 inner elements (16 bytes) x box_rows rows.
bool k_major_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || ((uintptr_t)base & 15) || (inner * 2) % 16) return false;
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {inner * 2};
  const cuuint32_t box[2] = {8, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// y = network(x) with the fused kernel; 1 when the shape does not suit it.
int predict_fused(swcs_mlp* m, const __nv_bfloat16* x, int64_t n, float* y) {
  const int D = m->p.d_in, W = m->p.width;
  if (D % 16 || D < 16 || D > 64 || W % 16 || W < 16 || W > 256 || ((uintptr_t)x & 15)) return 1;
  int dev = 0, nsm = 0, optin = 0;
  MCK(cudaGetDevice(&dev));
  MCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  MCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (mlp_fused_smem_bytes(D, W) > (size_t)optin) return 1;
  CUtensorMap tx, tw1, tw2;
  if (!k_major_map(&tx, x, (uint64_t)D, (uint64_t)n, 128) ||
      !k_major_map(&tw1, m->p.W1b, (uint64_t)D, (uint64_t)W, (uint32_t)W) ||
      !k_major_map(&tw2, m->p.W2b, (uint64_t)W, (uint64_t)W, (uint32_t)W))
    return 1;
  FusedArgs f{};
  f.M = n;
  f.d_in = D;
  f.width = W;
  f.b1 = m->p.master + m->p.off_b1;
  f.b2 = m->p.master + m->p.off_b2;
  f.w3 = m->p.w3b;
  f.b3 = m->p.master + m->p.off_b3;
  f.y = y;
  f.err = m->err_dev;
  const int64_t tiles = (n + 127) / 128;
  MCK(launch_mlp_fused(tx, tw1, tw2, f, (int)(tiles < nsm ? tiles : nsm), m->st));
  m->launches += 1;
  return SWCS_OK;
}

__global__ void add_b3_kernel(float* y, int64_t n, const float* b3) {
  const float b = *b3;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += b;
}

int add_b3(swcs_mlp* m, float* y, int64_t n) {
  add_b3_kernel<<<(int)((n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216), 256, 0, m->st>>>(y, n, m->p.master + m->p.off_b3);
  MCK(cudaGetLastError());
  m->launches += 1;
  return SWCS_OK;
}

int grads(swcs_mlp* m, const __nv_bfloat16* x, const float* t, int64_t n, double* d_loss) {
  const int W = m->p.width, D = m->p.d_in;
  int r;
  if ((r = ensure_rows(m, n))) return r;
  const int Bpad = (int)(((n + 31) / 32) * 32);
  MCK(cudaMemsetAsync(m->grad, 0, sizeof(float) * m->p.n_params, m->st));
  MCK(cudaMemsetAsync(m->loss, 0, sizeof(double), m->st));
  if ((r = forward(m, x, n, m->y)) || (r = add_b3(m, m->y, n))) return r;
  MCK(launch_mlp_dy(m->y, t, (int)n, m->dy, m->loss, m->st));
  MCK(launch_mlp_dz2(m->dy, m->p.w3b, m->H2, (int)n, W, m->dZ2, m->grad + m->p.off_w3, m->grad + m->p.off_b3, m->st));
  GemmArgs g3 = gemm(m, m->dZ2, W, m->p.W2tb, W, (int)n, W, W, kGemmF32);  // dH1 = dZ2 W2
  g3.out_f32 = m->dH1;
  g3.ldo = W;
  if ((r = run_gemm(m, g3, false))) return r;
  MCK(launch_mlp_dz1(m->dH1, m->H1, (size_t)n * W, m->dZ1, m->st));
  MCK(launch_mlp_colsum(m->dZ2, (int)n, W, m->grad + m->p.off_b2, m->st));
  MCK(launch_mlp_colsum(m->dZ1, (int)n, W, m->grad + m->p.off_b1, m->st));
  MCK(launch_mlp_transpose(m->dZ2, (int)n, W, Bpad, m->dZ2t, m->st));
  MCK(launch_mlp_transpose(m->H1, (int)n, W, Bpad, m->H1t, m->st));
  MCK(launch_mlp_transpose(m->dZ1, (int)n, W, Bpad, m->dZ1t, m->st));
  MCK(launch_mlp_transpose(x, (int)n, D, Bpad, m->Xt, m->st));
  GemmArgs g4 = gemm(m, m->dZ2t, Bpad, m->H1t, Bpad, W, W, Bpad, kGemmF32);  // dW2 = dZ2^T H1
  g4.out_f32 = m->grad + m->p.off_W2;
  g4.ldo = W;
  if ((r = run_gemm(m, g4, true))) return r;  // into the zeroed gradient
  GemmArgs g5 = gemm(m, m->dZ1t, Bpad, m->Xt, Bpad, W, D, Bpad, kGemmF32);  // dW1 = dZ1^T X
  g5.out_f32 = m->grad + m->p.off_W1;
  g5.ldo = D;
  if ((r = run_gemm(m, g5, true))) return r;
  m->launches += 12;
  if (d_loss) MCK(cudaMemcpyAsync(d_loss, m->loss, sizeof(double), cudaMemcpyDeviceToDevice, m->st));
  return SWCS_OK;
}

}  // namespace

extern "C" {

int swcs_mlp_create(swcs_mlp** out, void* stream, int d_in, int width) {
  if (!out) return SWCS_ERR_INVALID_ARG;
  *out = nullptr;
  if (d_in <= 0 || d_in % 32 || d_in > 256 || width < 32 || width > 256 || width % 32) return SWCS_ERR_INVALID_ARG;
  swcs_mlp* m = new swcs_mlp();
  m->st = (cudaStream_t)stream;
  MlpParams& p = m->p;
  p.d_in = d_in;
  p.width = width;
  p.off_W1 = 0;
  p.off_b1 = p.off_W1 + width * d_in;
  p.off_W2 = p.off_b1 + width;
  p.off_b2 = p.off_W2 + width * width;
  p.off_w3 = p.off_b2 + width;
  p.off_b3 = p.off_w3 + width;
  p.n_params = p.off_b3 + 1;
  if (dalloc(&p.master, p.n_params) || dalloc(&p.m, p.n_params) || dalloc(&p.v, p.n_params) ||
      dalloc(&m->grad, p.n_params) || dalloc(&m->loss, 1) || dalloc(&p.W1b, (size_t)width * d_in) ||
      dalloc(&p.W2b, (size_t)width * width) || dalloc(&p.W2tb, (size_t)width * width) || dalloc(&p.w3b, width) ||
      dalloc(&m->err_dev, 1)) {
    cudaGetLastError();
    swcs_mlp_destroy(m);
    return SWCS_ERR_OOM;
  }
  cudaMemset(p.master, 0, sizeof(float) * p.n_params);
  cudaMemset(p.m, 0, sizeof(float) * p.n_params);
  cudaMemset(p.v, 0, sizeof(float) * p.n_params);
  cudaMemset(m->err_dev, 0, sizeof(int));
  *out = m;
  return SWCS_OK;
}

int swcs_mlp_destroy(swcs_mlp* m) {
  if (!m) return SWCS_OK;
  cudaStreamSynchronize(m->st);
  free_scratch(m);
  void* bufs[] = {m->p.master, m->p.m, m->p.v, m->grad, m->loss, m->p.W1b, m->p.W2b, m->p.W2tb, m->p.w3b, m->err_dev};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete m;
  return SWCS_OK;
}

const char* swcs_mlp_last_error(const swcs_mlp* m) { return m ? m->err.c_str() : "no network"; }

int swcs_mlp_param_count(swcs_mlp* m, int64_t* n) {
  if (!m || !n) return SWCS_ERR_INVALID_ARG;
  *n = m->p.n_params;
  return SWCS_OK;
}

int swcs_mlp_set_params(swcs_mlp* m, const float* h) {
  if (!m || !h) return SWCS_ERR_INVALID_ARG;
  MCK(cudaMemcpyAsync(m->p.master, h, sizeof(float) * m->p.n_params, cudaMemcpyHostToDevice, m->st));
  MCK(cudaMemsetAsync(m->p.m, 0, sizeof(float) * m->p.n_params, m->st));
  MCK(cudaMemsetAsync(m->p.v, 0, sizeof(float) * m->p.n_params, m->st));
  MCK(launch_mlp_refresh(m->p, m->st));
  m->step = 0;
  MCK(cudaStreamSynchronize(m->st));
  return SWCS_OK;
}

int swcs_mlp_get_params(swcs_mlp* m, float* h) {
  if (!m || !h) return SWCS_ERR_INVALID_ARG;
  MCK(cudaMemcpyAsync(h, m->p.master, sizeof(float) * m->p.n_params, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  return SWCS_OK;
}

int swcs_mlp_forward_dev(swcs_mlp* m, const uint16_t* d_x, int64_t n, float* d_y) {
  if (!m || !d_x || !d_y || n <= 0) return SWCS_ERR_INVALID_ARG;
  int r;
  if ((r = ensure_rows(m, n))) return r;
  if ((r = forward(m, (const __nv_bfloat16*)d_x, n, d_y))) return r;
  return add_b3(m, d_y, n);
}

int swcs_mlp_predict_dev(swcs_mlp* m, const uint16_t* d_x, int64_t n, float* d_y) {
  if (!m || !d_x || !d_y || n <= 0 || n > ((int64_t)1 << 31)) return SWCS_ERR_INVALID_ARG;
  const int r = predict_fused(m, (const __nv_bfloat16*)d_x, n, d_y);
  if (r != 1) return r;
  return swcs_mlp_forward_dev(m, d_x, n, d_y);  // layer by layer, same result
}

int swcs_mlp_grad_dev(swcs_mlp* m, const uint16_t* d_x, const float* d_t, int64_t n, float* d_grad, double* d_loss) {
  if (!m || !d_x || !d_t || n <= 0) return SWCS_ERR_INVALID_ARG;
  int r = grads(m, (const __nv_bfloat16*)d_x, d_t, n, d_loss);
  if (r) return r;
  if (d_grad) MCK(cudaMemcpyAsync(d_grad, m->grad, sizeof(float) * m->p.n_params, cudaMemcpyDeviceToDevice, m->st));
  return SWCS_OK;
}

int swcs_mlp_train_step_dev(swcs_mlp* m, const uint16_t* d_x, const float* d_t, int64_t n, float lr, double* d_loss) {
  if (!m || !d_x || !d_t || n <= 0) return SWCS_ERR_INVALID_ARG;
  int r = grads(m, (const __nv_bfloat16*)d_x, d_t, n, d_loss);
  if (r) return r;
  m->step += 1;
  MCK(launch_mlp_adam(m->p, m->grad, lr, m->step, m->st));
  MCK(launch_mlp_refresh(m->p, m->st));
  m->launches += 2;
  return SWCS_OK;
}

int swcs_mlp_activations(swcs_mlp* m, uint16_t* h_H1, uint16_t* h_H2, float* h_y, int64_t n) {
  if (!m || n > m->cap) return SWCS_ERR_INVALID_ARG;
  const size_t W = (size_t)m->p.width;
  if (h_H1) MCK(cudaMemcpyAsync(h_H1, m->H1, n * W * 2, cudaMemcpyDeviceToHost, m->st));
  if (h_H2) MCK(cudaMemcpyAsync(h_H2, m->H2, n * W * 2, cudaMemcpyDeviceToHost, m->st));
  if (h_y) MCK(cudaMemcpyAsync(h_y, m->y, n * 4, cudaMemcpyDeviceToHost, m->st));
  MCK(cudaStreamSynchronize(m->st));
  int e = 0;
  MCK(cudaMemcpy(&e, m->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) return mfail(m, SWCS_ERR_TIMEOUT, "mlp: a tensor-core wait timed out");
  return SWCS_OK;
}

int swcs_mlp_set_option(swcs_mlp* m, const char* key, int64_t value) {
  if (!m) return SWCS_ERR_INVALID_ARG;
  if (!key) return mfail(m, SWCS_ERR_INVALID_ARG, "mlp_set_option: null key");
  const std::string k(key);
  if (k == "gemm_pipeline") {
    if (value != 0 && value != 1) return mfail(m, SWCS_ERR_INVALID_ARG, "gemm_pipeline must be 0 or 1");
    m->pipeline = value != 0;
    return SWCS_OK;
  }
  return mfail(m, SWCS_ERR_INVALID_ARG, "mlp_set_option: unknown key " + k);
}

int swcs_mlp_sync(swcs_mlp* m) {
  if (!m) return SWCS_ERR_INVALID_ARG;
  MCK(cudaStreamSynchronize(m->st));
  int e = 0;
  MCK(cudaMemcpy(&e, m->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) return mfail(m, SWCS_ERR_TIMEOUT, "mlp: a tensor-core wait timed out");
  return SWCS_OK;
}

int swcs_log_abs_dev(const double* d_g, int64_t n, float* d_t, void* stream) {
  if (!d_g || !d_t || n < 0) return SWCS_ERR_INVALID_ARG;
  return launch_log_abs(d_g, n, d_t, (cudaStream_t)stream) == cudaSuccess ? SWCS_OK : SWCS_ERR_CUDA;
}

}  // extern "C"
