// Per-query parameter model (an addition; the paper tunes alpha_q / cut and
// heap_factor globally, Section 5.3): MLP 64 -> 128 -> 64 -> 2 with ReLU,
// fp32 weights and bf16 activations.  Outputs map to
//   cut = clamp(round(3 + 27 * sigmoid(o0)), 3, 30)
//   heap_factor = 0.5 + 0.5 * sigmoid(o1)
// Training: loss = mean over rows of sum_j (sigmoid(o_j) - t_j)^2, Adam.
#include <cuda_bf16.h>

#include "search_impl.h"

namespace seismic {

namespace {

constexpr int IN = SEISMIC_MLP_IN, H1 = SEISMIC_MLP_H1, H2 = SEISMIC_MLP_H2, OUT = 2;
constexpr int OW1 = 0, OB1 = OW1 + H1 * IN, OW2 = OB1 + H1, OB2 = OW2 + H2 * H1, OW3 = OB2 + H2, OB3 = OW3 + OUT * H2;
static_assert(OB3 + OUT == SEISMIC_MLP_PARAMS, "parameter packing");
constexpr int kRows = 32;  // rows per CTA
constexpr int kNT = 128;

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + __expf(-x)); }

struct MlpSmem {
  float w[SEISMIC_MLP_PARAMS];
  float a0[kRows][IN];
  float z1[kRows][H1];  // pre-activation
  float a1[kRows][H1];  // bf16-rounded ReLU
  float z2[kRows][H2];
  float a2[kRows][H2];
  float o[kRows][OUT];
};

// forward for rows [r0, r0 + nr) held in shared memory
__device__ void mlp_fwd(MlpSmem &s, const float *feat, uint64_t r0, int nr) {
  const int tid = threadIdx.x;
  for (int i = tid; i < kRows * IN; i += kNT) {
    int r = i / IN, f = i % IN;
    s.a0[r][f] = r < nr ? bfr(feat[(r0 + r) * IN + f]) : 0.0f;
  }
  __syncthreads();
  for (int i = tid; i < kRows * H1; i += kNT) {
    int r = i / H1, m = i % H1;
    float z = s.w[OB1 + m];
    const float *w = s.w + OW1 + m * IN;
    for (int f = 0; f < IN; f++) z = fmaf(w[f], s.a0[r][f], z);
    s.z1[r][m] = z;
    s.a1[r][m] = bfr(fmaxf(z, 0.0f));
  }
  __syncthreads();
  for (int i = tid; i < kRows * H2; i += kNT) {
    int r = i / H2, m = i % H2;
    float z = s.w[OB2 + m];
    const float *w = s.w + OW2 + m * H1;
    for (int f = 0; f < H1; f++) z = fmaf(w[f], s.a1[r][f], z);
    s.z2[r][m] = z;
    s.a2[r][m] = bfr(fmaxf(z, 0.0f));
  }
  __syncthreads();
  for (int i = tid; i < kRows * OUT; i += kNT) {
    int r = i / OUT, j = i % OUT;
    float z = s.w[OB3 + j];
    const float *w = s.w + OW3 + j * H2;
    for (int f = 0; f < H2; f++) z = fmaf(w[f], s.a2[r][f], z);
    s.o[r][j] = z;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kNT) k_mlp_forward(const float *__restrict__ w, const float *__restrict__ feat,
                                                      uint64_t n, float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MlpSmem &s = *reinterpret_cast<MlpSmem *>(smraw);
  for (int i = threadIdx.x; i < SEISMIC_MLP_PARAMS; i += kNT) s.w[i] = w[i];
  __syncthreads();
  for (uint64_t r0 = (uint64_t)blockIdx.x * kRows; r0 < n; r0 += (uint64_t)gridDim.x * kRows) {
    int nr = (int)((n - r0) < (uint64_t)kRows ? (n - r0) : (uint64_t)kRows);
    mlp_fwd(s, feat, r0, nr);
    for (int i = threadIdx.x; i < nr * OUT; i += kNT) out[r0 * OUT + i] = s.o[i / OUT][i % OUT];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kNT) k_mlp_params(const float *__restrict__ w, const float *__restrict__ feat,
                                                     uint64_t n, uint32_t cut_fb, float hf_fb,
                                                     uint32_t *__restrict__ q_cut, float *__restrict__ q_hf) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MlpSmem &s = *reinterpret_cast<MlpSmem *>(smraw);
  for (int i = threadIdx.x; i < SEISMIC_MLP_PARAMS; i += kNT) s.w[i] = w[i];
  __syncthreads();
  for (uint64_t r0 = (uint64_t)blockIdx.x * kRows; r0 < n; r0 += (uint64_t)gridDim.x * kRows) {
    int nr = (int)((n - r0) < (uint64_t)kRows ? (n - r0) : (uint64_t)kRows);
    mlp_fwd(s, feat, r0, nr);
    for (int r = threadIdx.x; r < nr; r += kNT) {
      float o0 = s.o[r][0], o1 = s.o[r][1];
      uint32_t c = cut_fb;
      float h = hf_fb;
      if (isfinite(o0) && isfinite(o1)) {  // fixed parameters are the fallback
        c = (uint32_t)min(30.0f, max(3.0f, rintf(3.0f + 27.0f * sigm(o0))));
        h = 0.5f + 0.5f * sigm(o1);
      }
      q_cut[r0 + r] = c;
      q_hf[r0 + r] = h;
    }
    __syncthreads();
  }
}

// forward + backward; gradients accumulated with atomics into g (zeroed by caller)
__global__ void __launch_bounds__(kNT) k_mlp_grad(const float *__restrict__ w, const float *__restrict__ feat,
                                                   const float *__restrict__ tgt, uint64_t n, float *__restrict__ g,
                                                   float *__restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MlpSmem &s = *reinterpret_cast<MlpSmem *>(smraw);
  float *gl = reinterpret_cast<float *>(smraw + sizeof(MlpSmem));  // local gradient, SEISMIC_MLP_PARAMS
  __shared__ float dz2[kRows][H2], dz1[kRows][H1], dzo[kRows][OUT];
  __shared__ float lsum;
  const int tid = threadIdx.x;
  for (int i = tid; i < SEISMIC_MLP_PARAMS; i += kNT) {
    s.w[i] = w[i];
    gl[i] = 0.0f;
  }
  if (tid == 0) lsum = 0.0f;
  __syncthreads();
  const float inv_n = 1.0f / (float)n;
  for (uint64_t r0 = (uint64_t)blockIdx.x * kRows; r0 < n; r0 += (uint64_t)gridDim.x * kRows) {
    const int nr = (int)((n - r0) < (uint64_t)kRows ? (n - r0) : (uint64_t)kRows);
    mlp_fwd(s, feat, r0, nr);
    for (int i = tid; i < kRows * OUT; i += kNT) {
      int r = i / OUT, j = i % OUT;
      float d = 0.0f;
      if (r < nr) {
        float sg = sigm(s.o[r][j]), e = sg - tgt[(r0 + r) * OUT + j];
        atomicAdd(&lsum, e * e * inv_n);
        d = 2.0f * e * sg * (1.0f - sg) * inv_n;
      }
      dzo[r][j] = d;
    }
    __syncthreads();
    for (int i = tid; i < kRows * H2; i += kNT) {
      int r = i / H2, m = i % H2;
      float d = 0.0f;
      for (int j = 0; j < OUT; j++) d = fmaf(s.w[OW3 + j * H2 + m], dzo[r][j], d);
      dz2[r][m] = s.z2[r][m] > 0.0f ? d : 0.0f;
    }
    __syncthreads();
    for (int i = tid; i < kRows * H1; i += kNT) {
      int r = i / H1, m = i % H1;
      float d = 0.0f;
      for (int j = 0; j < H2; j++) d = fmaf(s.w[OW2 + j * H1 + m], dz2[r][j], d);
      dz1[r][m] = s.z1[r][m] > 0.0f ? d : 0.0f;
    }
    __syncthreads();
    // weight gradients: each thread owns parameters, summing over the CTA's rows
    for (int p = tid; p < SEISMIC_MLP_PARAMS; p += kNT) {
      float acc = 0.0f;
      if (p < OB1) {
        int m = p / IN, f = p % IN;
        for (int r = 0; r < nr; r++) acc = fmaf(dz1[r][m], s.a0[r][f], acc);
      } else if (p < OW2) {
        int m = p - OB1;
        for (int r = 0; r < nr; r++) acc += dz1[r][m];
      } else if (p < OB2) {
        int q = p - OW2, m = q / H1, f = q % H1;
        for (int r = 0; r < nr; r++) acc = fmaf(dz2[r][m], s.a1[r][f], acc);
      } else if (p < OW3) {
        int m = p - OB2;
        for (int r = 0; r < nr; r++) acc += dz2[r][m];
      } else if (p < OB3) {
        int q = p - OW3, j = q / H2, f = q % H2;
        for (int r = 0; r < nr; r++) acc = fmaf(dzo[r][j], s.a2[r][f], acc);
      } else {
        int j = p - OB3;
        for (int r = 0; r < nr; r++) acc += dzo[r][j];
      }
      gl[p] += acc;
    }
    __syncthreads();
  }
  for (int p = tid; p < SEISMIC_MLP_PARAMS; p += kNT) atomicAdd(&g[p], gl[p]);
  if (tid == 0) atomicAdd(loss, lsum);
}

__global__ void k_adam(float *w, const float *g, float *m, float *v, float lr, float b1c, float b2c) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < SEISMIC_MLP_PARAMS; i += gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / b1c) / (sqrtf(vi / b2c) + eps);
  }
}

// features: one warp per query
__global__ void k_features(const uint64_t *__restrict__ ip, const uint16_t *__restrict__ terms,
                           const float *__restrict__ vals, uint32_t nq, const uint32_t *__restrict__ list_ptr,
                           const uint32_t *__restrict__ blk_ptr, uint32_t dim, float *__restrict__ feat) {
  const int lane = threadIdx.x & 31;
  const uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= nq) return;
  const uint64_t b = ip[q], e = ip[q + 1];
  float *f = feat + (size_t)q * IN;
  for (int i = lane; i < IN; i += 32) f[i] = 0.0f;
  __syncwarp();
  uint32_t nz = 0;
  float l1 = 0.0f, l2 = 0.0f;
  for (uint64_t p = b + lane; p < e; p += 32) {
    float v = vals[p];
    if (v == 0.0f) continue;
    nz++;
    l1 += fabsf(v);
    l2 = fmaf(v, v, l2);
    const uint16_t t = terms[p];
    uint32_t r = 0;  // rank by (value desc, term asc) among nonzeros
    for (uint64_t j = b; j < e; j++) {
      float vj = vals[j];
      if (vj == 0.0f) continue;
      r += (vj > v || (vj == v && terms[j] < t)) ? 1u : 0u;
    }
    if (r < 16 && t < dim) {
      f[1 + r] = v;
      f[17 + r] = __logf(1.0f + (float)(list_ptr[t + 1] - list_ptr[t]));
      f[33 + r] = __logf(1.0f + (float)(blk_ptr[t + 1] - blk_ptr[t]));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    nz += __shfl_xor_sync(0xffffffffu, nz, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    l2 += __shfl_xor_sync(0xffffffffu, l2, o);
  }
  if (lane == 0) {
    f[0] = __logf(1.0f + (float)nz);
    f[49] = l1;
    f[50] = sqrtf(l2);
  }
}

size_t mlp_smem(bool grad) { return sizeof(MlpSmem) + (grad ? SEISMIC_MLP_PARAMS * 4 : 0); }

int set_attr(const void *fn, size_t smem) {
  SZ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return SEISMIC_OK;
}

}  // namespace

int launch_features(const uint64_t *ip, const uint16_t *t, const float *v, uint32_t nq, const uint32_t *list_ptr,
                    const uint32_t *blk_ptr, uint32_t dim, float *feat, cudaStream_t st) {
  if (!nq) return SEISMIC_OK;
  const uint32_t warps_per_block = 8;
  k_features<<<(nq + warps_per_block - 1) / warps_per_block, warps_per_block * 32, 0, st>>>(ip, t, v, nq, list_ptr,
                                                                                           blk_ptr, dim, feat);
  SZ_CUDA(cudaGetLastError());
  return SEISMIC_OK;
}

int launch_mlp_params(const float *w, const float *feat, uint32_t n, uint32_t cut_fb, float hf_fb, uint32_t *q_cut,
                      float *q_hf, cudaStream_t st) {
  if (!n) return SEISMIC_OK;
  size_t sm = mlp_smem(false);
  int rc = set_attr((const void *)k_mlp_params, sm);
  if (rc) return rc;
  uint32_t grid = std::min<uint32_t>((n + kRows - 1) / kRows, 1024);
  k_mlp_params<<<grid, kNT, sm, st>>>(w, feat, n, cut_fb, hf_fb, q_cut, q_hf);
  SZ_CUDA(cudaGetLastError());
  return SEISMIC_OK;
}

int mlp_forward_impl(const float *w, const float *feat, uint64_t n, float *out, cudaStream_t st) {
  if (!w || !feat || !out) return fail(SEISMIC_EINVAL, "NULL argument");
  if (!n) return SEISMIC_OK;
  size_t sm = mlp_smem(false);
  int rc = set_attr((const void *)k_mlp_forward, sm);
  if (rc) return rc;
  uint32_t grid = (uint32_t)std::min<uint64_t>((n + kRows - 1) / kRows, 1024);
  k_mlp_forward<<<grid, kNT, sm, st>>>(w, feat, n, out);
  SZ_CUDA(cudaGetLastError());
  return SEISMIC_OK;
}

int mlp_train_step_impl(float *w, float *g, float *m, float *v, const float *feat, const float *tgt, uint64_t n,
                        float lr, uint32_t step, float *loss, cudaStream_t st) {
  if (!w || !g || !m || !v || !feat || !tgt || !loss) return fail(SEISMIC_EINVAL, "NULL argument");
  if (!n || step == 0) return fail(SEISMIC_EINVAL, "n and step must be >= 1");
  size_t sm = mlp_smem(true);
  int rc = set_attr((const void *)k_mlp_grad, sm);
  if (rc) return rc;
  SZ_CUDA(cudaMemsetAsync(g, 0, SEISMIC_MLP_PARAMS * 4, st));
  SZ_CUDA(cudaMemsetAsync(loss, 0, 4, st));
  uint32_t grid = (uint32_t)std::min<uint64_t>((n + kRows - 1) / kRows, 304);
  k_mlp_grad<<<grid, kNT, sm, st>>>(w, feat, tgt, n, g, loss);
  SZ_CUDA(cudaGetLastError());
  float b1c = 1.0f - powf(0.9f, (float)step), b2c = 1.0f - powf(0.999f, (float)step);
  k_adam<<<(SEISMIC_MLP_PARAMS + 255) / 256, 256, 0, st>>>(w, g, m, v, lr, b1c, b2c);
  SZ_CUDA(cudaGetLastError());
  return SEISMIC_OK;
}

}  // namespace seismic

using namespace seismic;

extern "C" {

int seismic_set_mlp(seismic_index *ix, const float *weights, uint64_t n_floats) {
  if (!ix || !weights) return fail(SEISMIC_EINVAL, "NULL argument");
  if (n_floats != SEISMIC_MLP_PARAMS) return fail(SEISMIC_EINVAL, "MLP weights: wrong count");
  for (uint64_t i = 0; i < n_floats; i++)
    if (!std::isfinite(weights[i])) return fail(SEISMIC_EINVAL, "MLP weights: non-finite value");
  SZ_CUDA(cudaSetDevice(ix->device));
  int rc = ix->mlp.alloc(n_floats * 4);
  if (rc) return rc;
  SZ_CUDA(cudaMemcpy(ix->mlp.p, weights, n_floats * 4, cudaMemcpyHostToDevice));
  ix->has_mlp = 1;
  return SEISMIC_OK;
}

int seismic_query_features(seismic_index *ix, const seismic_csr *queries, float *features, int32_t on_device,
                           void *stream) {
  if (!ix || !queries || !features) return fail(SEISMIC_EINVAL, "NULL argument");
  if (queries->n_rows == 0) return SEISMIC_OK;
  if (queries->dim != ix->dim) return fail(SEISMIC_EINVAL, "queries: dim differs from the index");
  SZ_CUDA(cudaSetDevice(ix->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t nq = queries->n_rows;
  const uint64_t *ip = queries->indptr;
  const uint16_t *t = queries->terms;
  const float *v = queries->vals;
  DevBuf stage;
  if (!queries->on_device) {
    int rc = validate_host_csr(queries, "queries", ix->dim);
    if (rc) return rc;
    uint64_t nnz = queries->indptr[nq];
    size_t b_ip = (nq + 1) * 8, b_t = ((nnz * 2 + 15) / 16) * 16;
    if ((rc = stage.alloc(b_ip + b_t + nnz * 4 + 16))) return rc;
    uint8_t *base = stage.as<uint8_t>();
    SZ_CUDA(cudaMemcpyAsync(base, queries->indptr, b_ip, cudaMemcpyHostToDevice, st));
    if (nnz) {
      SZ_CUDA(cudaMemcpyAsync(base + b_ip, queries->terms, nnz * 2, cudaMemcpyHostToDevice, st));
      SZ_CUDA(cudaMemcpyAsync(base + b_ip + b_t, queries->vals, nnz * 4, cudaMemcpyHostToDevice, st));
    }
    ip = reinterpret_cast<const uint64_t *>(base);
    t = reinterpret_cast<const uint16_t *>(base + b_ip);
    v = reinterpret_cast<const float *>(base + b_ip + b_t);
  }
  float *dfeat = features;
  DevBuf fo;
  if (!on_device) {
    int rc = fo.alloc(nq * SEISMIC_MLP_IN * 4);
    if (rc) return rc;
    dfeat = fo.as<float>();
  }
  int rc = launch_features(ip, t, v, (uint32_t)nq, ix->list_ptr.as<uint32_t>(), ix->blk_ptr.as<uint32_t>(), ix->dim,
                           dfeat, st);
  if (rc) return rc;
  if (!on_device) {
    SZ_CUDA(cudaMemcpyAsync(features, dfeat, nq * SEISMIC_MLP_IN * 4, cudaMemcpyDeviceToHost, st));
  }
  SZ_CUDA(cudaStreamSynchronize(st));
  return SEISMIC_OK;
}

int seismic_mlp_forward(const float *weights, const float *features, uint64_t n, float *out, void *stream) {
  return mlp_forward_impl(weights, features, n, out, reinterpret_cast<cudaStream_t>(stream));
}

int seismic_mlp_train_step(float *weights, float *grads, float *adam_m, float *adam_v, const float *features,
                           const float *targets, uint64_t n, float lr, uint32_t step, float *loss_out, void *stream) {
  return mlp_train_step_impl(weights, grads, adam_m, adam_v, features, targets, n, lr, step, loss_out,
                             reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
