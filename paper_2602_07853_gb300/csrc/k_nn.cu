// Learned preconditioner: a 3-layer 3x3x3 convolutional network on the node
// grid (3 -> 16 -> 16 -> 3 channels, ReLU on the hidden layers, no biases),
// used inside flexible CG as z = D^-1 r + s D^-1/2 NN(D^-1/2 r / s), s the RMS
// of D^-1/2 r over free DOFs, and trained on residual / error pairs of the
// method's own Newton systems with the loss one minus the H-cosine of the
// preconditioned residual and the error e = H^-1 r,
//   L = 1 - z^T r / sqrt(z^T H z * e^T H e).
//
// Convolutions are BF16 implicit GEMMs on tensor cores (mma.sync m16n8k16,
// FP32 accumulation): one CTA per 8^3 brick, the 10^3 halo block of the
// input activations staged in shared memory (rows of 16 channels, 16-byte
// halves swizzled against bank conflicts) and fed to ldmatrix with one row
// address per node, so a tap is just a shifted set of row addresses.
// Channels are padded to 16.  Backward-data is the same convolution with the
// taps mirrored and each tap's weight matrix transposed; the weight gradient
// is an mma over the brick's nodes (ldmatrix.trans for both operands) with
// per-brick partials summed in a fixed order.
#include <cuda_bf16.h>

#include "mpml_internal.cuh"

namespace mpml {

constexpr int NNC = 16;                    // padded channels
constexpr int NN_LAYER = 27 * NNC * NNC;   // padded weights per layer
constexpr int HALO_N = 1000;               // 10^3 nodes
constexpr int HALO_BYTES = HALO_N * 32;    // 16 bf16 per node
constexpr int W_BYTES = NN_LAYER * 2;      // 13824

__host__ __device__ inline int nn_cin(int l) { return l == 0 ? 3 : 16; }
__host__ __device__ inline int nn_cout(int l) { return l == 2 ? 3 : 16; }

// ---------------------------------------------------------------------------
// PTX helpers (sm_80+ warp-level tensor core path, valid on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float c[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// byte offset of 16-byte half `c` of row `h` (rows of 32 bytes, halves
// swapped every 4 rows so the 8 rows of an ldmatrix phase hit distinct banks)
__device__ __forceinline__ unsigned row_off(int h, int c) { return (unsigned)(h * 32 + ((c ^ ((h >> 2) & 1)) << 4)); }

// stage the 10^3 halo block of a [brick][512][16] bf16 activation into smem
__device__ __forceinline__ void stage_halo(const __nv_bfloat16* __restrict__ act, int id, const int* s_nbr,
                                           unsigned char* sm) {
  for (int e = threadIdx.x; e < HALO_N * 2; e += blockDim.x) {
    const int h = e >> 1, c = e & 1;
    const int hx = h % 10, hy = (h / 10) % 10, hz = h / 100;
    const int nx = hx - 1, ny = hy - 1, nz = hz - 1;
    const int bx = nx < 0 ? -1 : (nx > 7 ? 1 : 0), by = ny < 0 ? -1 : (ny > 7 ? 1 : 0),
              bz = nz < 0 ? -1 : (nz > 7 ? 1 : 0);
    const int t = (bx | by | bz) == 0 ? id : s_nbr[nbr_index(bx, by, bz)];
    uint4 v = make_uint4(0, 0, 0, 0);
    if (t >= 0) {
      const int l = ((nz & 7) * 8 + (ny & 7)) * 8 + (nx & 7);
      v = reinterpret_cast<const uint4*>(act + ((int64_t)t * BV + l) * NNC)[c];
    }
    *reinterpret_cast<uint4*>(sm + row_off(h, c)) = v;
  }
}

// ---------------------------------------------------------------------------
// Convolution: out[i][n] = sum_t sum_k W[t][n][k] in[i + d_t][k]
// MODE 0: hidden layer  -> bf16, ReLU, zero off DOF nodes
// MODE 1: output layer  -> fp32 y[brick][3][512] (node layout), zero off free DOFs
// MODE 2: backward-data -> bf16, kept where the forward activation `ref` > 0
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_conv(const __nv_bfloat16* __restrict__ in,
                                              const __nv_bfloat16* __restrict__ W, const int* __restrict__ nbr,
                                              const uint8_t* __restrict__ nflag,
                                              const __nv_bfloat16* __restrict__ ref, __nv_bfloat16* out_bf,
                                              float* out_f) {
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char* ws = sm + HALO_BYTES;
  __shared__ int s_nbr[NBR];
  const int id = blockIdx.x;
  if (threadIdx.x < NBR) s_nbr[threadIdx.x] = nbr[id * NBR + threadIdx.x];
  __syncthreads();
  stage_halo(in, id, s_nbr, sm);
  for (int e = threadIdx.x; e < 27 * 16 * 2; e += blockDim.x) {
    const int rr = e >> 1, c = e & 1;  // row = t * 16 + n
    *reinterpret_cast<uint4*>(ws + row_off(rr, c)) = reinterpret_cast<const uint4*>(W + rr * NNC)[c];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned sbase = su32(sm), wbase = su32(ws);
  for (int mt = warp * 4; mt < warp * 4 + 4; ++mt) {
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    const int la = 16 * mt + (lane & 15);
    const int lx = la & 7, ly = (la >> 3) & 7, lz = la >> 6;
    const int ca = lane >> 4;
    const int nb_row = (lane & 7) + ((lane >> 4) << 3), cb = (lane >> 3) & 1;
#pragma unroll 3
    for (int t = 0; t < 27; ++t) {
      const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
      const int h = ((lz + 1 + dz) * 10 + (ly + 1 + dy)) * 10 + (lx + 1 + dx);
      unsigned a0, a1, a2, a3, b0, b1, b2, b3;
      ldsm_x4(sbase + row_off(h, ca), a0, a1, a2, a3);
      const int rr = t * 16 + nb_row;
      ldsm_x4(wbase + row_off(rr, cb), b0, b1, b2, b3);
      mma_bf16(acc[0], a0, a1, a2, a3, b0, b1);
      mma_bf16(acc[1], a0, a1, a2, a3, b2, b3);
    }
    const int g = lane >> 2, tg = lane & 3;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int l = 16 * mt + g + 8 * half;
      const uint8_t f = nflag[(int64_t)id * BV + l];
      const bool dof = f & NF_DOF, fre = dof && !(f & NF_FIXED);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int n = 8 * j + 2 * tg;
        float v0 = acc[j][2 * half], v1 = acc[j][2 * half + 1];
        if (MODE == 0) {
          v0 = dof ? fmaxf(v0, 0.f) : 0.f;
          v1 = dof ? fmaxf(v1, 0.f) : 0.f;
          *reinterpret_cast<__nv_bfloat162*>(out_bf + ((int64_t)id * BV + l) * NNC + n) = __floats2bfloat162_rn(v0, v1);
        } else if (MODE == 2) {
          const __nv_bfloat162 rv = *reinterpret_cast<const __nv_bfloat162*>(ref + ((int64_t)id * BV + l) * NNC + n);
          v0 = (dof && __bfloat162float(rv.x) > 0.f) ? v0 : 0.f;
          v1 = (dof && __bfloat162float(rv.y) > 0.f) ? v1 : 0.f;
          *reinterpret_cast<__nv_bfloat162*>(out_bf + ((int64_t)id * BV + l) * NNC + n) = __floats2bfloat162_rn(v0, v1);
        } else {
          if (j == 0) {
            if (n < 3) out_f[((int64_t)id * 3 + n) * BV + l] = fre ? v0 : 0.f;
            if (n + 1 < 3) out_f[((int64_t)id * 3 + n + 1) * BV + l] = fre ? v1 : 0.f;
          }
        }
      }
    }
  }
}

// Weight gradient of one layer: part[brick][t][n][k] = sum_{i in brick} g[i][n] a[i + d_t][k]
__global__ void __launch_bounds__(256) k_conv_wgrad(const __nv_bfloat16* __restrict__ a,
                                                    const __nv_bfloat16* __restrict__ g,
                                                    const int* __restrict__ nbr, float* __restrict__ part) {
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char* gs = sm + HALO_BYTES;  // [512][32 B]
  __shared__ int s_nbr[NBR];
  const int id = blockIdx.x;
  if (threadIdx.x < NBR) s_nbr[threadIdx.x] = nbr[id * NBR + threadIdx.x];
  __syncthreads();
  stage_halo(a, id, s_nbr, sm);
  for (int e = threadIdx.x; e < BV * 2; e += blockDim.x) {
    const int l = e >> 1, c = e & 1;
    *reinterpret_cast<uint4*>(gs + row_off(l, c)) = reinterpret_cast<const uint4*>(g + ((int64_t)id * BV + l) * NNC)[c];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned sbase = su32(sm), gbase = su32(gs);
  for (int t = warp; t < 27; t += 8) {
    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    for (int ks = 0; ks < 32; ++ks) {
      // A (n x nodes) from g: matrices (nodes 0-7 | n 0-7), (nodes 0-7 | n 8-15),
      // (nodes 8-15 | n 0-7), (nodes 8-15 | n 8-15), transposed on load
      const int la = 16 * ks + (lane & 7) + ((lane >> 4) << 3);
      const int ca = (lane >> 3) & 1;
      unsigned a0, a1, a2, a3;
      ldsm_x4_t(gbase + row_off(la, ca), a0, a1, a2, a3);
      // B (nodes x k) from the shifted halo rows: (nodes 0-7 | k 0-7), (nodes 8-15 | k 0-7),
      // (nodes 0-7 | k 8-15), (nodes 8-15 | k 8-15)
      const int lb = 16 * ks + (lane & 15);
      const int cb = lane >> 4;
      const int lx = lb & 7, ly = (lb >> 3) & 7, lz = lb >> 6;
      const int h = ((lz + 1 + dz) * 10 + (ly + 1 + dy)) * 10 + (lx + 1 + dx);
      unsigned b0, b1, b2, b3;
      ldsm_x4_t(sbase + row_off(h, cb), b0, b1, b2, b3);
      mma_bf16(acc[0], a0, a1, a2, a3, b0, b1);
      mma_bf16(acc[1], a0, a1, a2, a3, b2, b3);
    }
    const int gq = lane >> 2, tg = lane & 3;
    float* dst = part + ((int64_t)id * 27 + t) * NNC * NNC;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int k = 8 * j + 2 * tg;
      dst[gq * NNC + k] = acc[j][0];
      dst[gq * NNC + k + 1] = acc[j][1];
      dst[(gq + 8) * NNC + k] = acc[j][2];
      dst[(gq + 8) * NNC + k + 1] = acc[j][3];
    }
  }
}

// sum the per-brick partials (fixed order): out[e] += scale * sum_b part[b][e]
__global__ void k_wgrad_reduce(const float* __restrict__ part, int nb, float scale, float* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NN_LAYER) return;
  double s = 0;
  for (int b = 0; b < nb; ++b) s += (double)part[(int64_t)b * NN_LAYER + e];
  out[e] += scale * (float)s;
}

// master FP32 weights [3][27][16][16] (n, k) -> bf16 forward copy and the
// backward-data copy Wb[l][t][k][n] = W[l][26 - t][n][k]
__global__ void k_nn_weights(const float* __restrict__ master, __nv_bfloat16* wf, __nv_bfloat16* wb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 * NN_LAYER) return;
  const int l = e / NN_LAYER, r = e % NN_LAYER;
  const int t = r / (NNC * NNC), n = (r / NNC) % NNC, k = r % NNC;
  wf[e] = __float2bfloat16_rn(master[e]);
  wb[(int64_t)l * NN_LAYER + ((26 - t) * NNC + k) * NNC + n] = __float2bfloat16_rn(master[e]);
}

// network input: x = sqrt(D^-1) r / s on free DOFs (channels 0..2, rest 0)
__global__ void __launch_bounds__(512) k_nn_input(const float* __restrict__ r, const float* __restrict__ dinv,
                                                  const double* s_ptr, __nv_bfloat16* x) {
  const int id = blockIdx.x, l = threadIdx.x;
  const double s = *s_ptr;
  const float is = s > 0 ? (float)(1.0 / s) : 0.f;
  __align__(16) __nv_bfloat16 v[NNC];
#pragma unroll
  for (int c = 0; c < NNC; ++c) v[c] = __float2bfloat16_rn(0.f);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int64_t o = ((int64_t)id * 3 + c) * BV + l;
    const float di = dinv[o];
    v[c] = __float2bfloat16_rn(di > 0.f ? sqrtf(di) * r[o] * is : 0.f);
  }
  uint4* dst = reinterpret_cast<uint4*>(x + ((int64_t)id * BV + l) * NNC);
  dst[0] = reinterpret_cast<const uint4*>(v)[0];
  dst[1] = reinterpret_cast<const uint4*>(v)[1];
}

// z = D^-1 r + s sqrt(D^-1) y, with FP64 sums z^T q and z^T r (FCG) in partials
__global__ void __launch_bounds__(512) k_nn_combine(const float* __restrict__ r, const float* __restrict__ dinv,
                                                    const float* __restrict__ y, const float* __restrict__ q,
                                                    const double* s_ptr, float* z, double* part) {
  const int id = blockIdx.x, l = threadIdx.x;
  const float s = (float)*s_ptr;
  float zq = 0.f, zr = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int64_t o = ((int64_t)id * 3 + c) * BV + l;
    const float di = dinv[o];
    float zv = 0.f;
    if (di > 0.f) zv = di * r[o] + s * sqrtf(di) * y[o];
    z[o] = zv;
    if (q) zq += zv * q[o];
    zr += zv * r[o];
  }
  if (part) {
    __shared__ double red[2][16];
    double a = zq, b = zr;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((l & 31) == 0) {
      red[0][l >> 5] = a;
      red[1][l >> 5] = b;
    }
    __syncthreads();
    if (l == 0) {
      double sa = 0, sb = 0;
      for (int w = 0; w < 16; ++w) {
        sa += red[0][w];
        sb += red[1][w];
      }
      part[2 * id] = sa;
      part[2 * id + 1] = sb;
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct NNBufs {
  __nv_bfloat16 *wf, *wb, *x, *h1, *h2, *g, *g2;
  float *master, *y, *part, *grad, *adam_m, *adam_v;
};

static NNBufs nn_bufs(mpml_ctx_s* c) {
  NNBufs b;
  char* w = (char*)c->nnw.p;
  b.master = (float*)w;
  b.grad = b.master + 3 * NN_LAYER;
  b.adam_m = b.grad + 3 * NN_LAYER;
  b.adam_v = b.adam_m + 3 * NN_LAYER;
  b.wf = (__nv_bfloat16*)(b.adam_v + 3 * NN_LAYER);
  b.wb = b.wf + 3 * NN_LAYER;
  const int64_t ns = c->nb * BV;
  __nv_bfloat16* a = (__nv_bfloat16*)c->nnact.p;
  b.x = a;
  b.h1 = a + ns * NNC;
  b.h2 = a + 2 * ns * NNC;
  b.g = a + 3 * ns * NNC;
  b.g2 = a + 4 * ns * NNC;
  b.y = (float*)c->nny.p;
  b.part = (float*)c->nnpart.p;
  return b;
}

int nn_ensure(mpml_ctx_s* c) {
  int rc;
  const size_t wbytes = 4 * sizeof(float) * 3 * NN_LAYER + 2 * sizeof(__nv_bfloat16) * 3 * NN_LAYER;
  const bool fresh = c->nnw.p == nullptr;
  if ((rc = ensure(c->nnw, wbytes))) return rc;
  if (fresh) cudaMemsetAsync(c->nnw.p, 0, wbytes, c->s);
  const int64_t ns = c->nb * BV;
  if ((rc = ensure(c->nnact, sizeof(__nv_bfloat16) * 5 * NNC * (ns ? ns : 1))) ||
      (rc = ensure(c->nny, sizeof(float) * 3 * (ns ? ns : 1))) ||
      (rc = ensure(c->nnpart, sizeof(float) * (size_t)NN_LAYER * (c->nb ? c->nb : 1))) ||
      (rc = ensure(c->nz, sizeof(float) * 3 * (ns ? ns : 1))))
    return rc;
  return MPML_OK;
}

// shared-memory limits of the convolution kernels, once per device
static void set_conv_attrs() {
  launch_fit((const void*)k_conv<0>, 256, HALO_BYTES + W_BYTES, LS_CONV + 0, nullptr);
  launch_fit((const void*)k_conv<1>, 256, HALO_BYTES + W_BYTES, LS_CONV + 1, nullptr);
  launch_fit((const void*)k_conv<2>, 256, HALO_BYTES + W_BYTES, LS_CONV + 2, nullptr);
  launch_fit((const void*)k_conv_wgrad, 256, HALO_BYTES + BV * 32, LS_CONV + 3, nullptr);
}

int nn_refresh_weights(mpml_ctx_s* c) {
  NNBufs b = nn_bufs(c);
  k_nn_weights<<<div_up(3 * NN_LAYER, 256), 256, 0, c->s>>>(b.master, b.wf, b.wb);
  c->launches++;
  return cuda_status(cudaGetLastError());
}

// forward network on x (already in b.x): h1, h2 (bf16) and y (fp32)
void nn_forward(mpml_ctx_s* c) {
  set_conv_attrs();
  NNBufs b = nn_bufs(c);
  const unsigned nb = (unsigned)c->nb;
  const size_t smem = HALO_BYTES + W_BYTES;
  const uint8_t* nf = (const uint8_t*)c->nflag.p;
  const int* nbr = (const int*)c->nbr.p;
  k_conv<0><<<nb, 256, smem, c->s>>>(b.x, b.wf, nbr, nf, nullptr, b.h1, nullptr);
  k_conv<0><<<nb, 256, smem, c->s>>>(b.h1, b.wf + NN_LAYER, nbr, nf, nullptr, b.h2, nullptr);
  k_conv<1><<<nb, 256, smem, c->s>>>(b.h2, b.wf + 2 * NN_LAYER, nbr, nf, nullptr, nullptr, b.y);
  c->launches += 3;
}

// preconditioner application z = D^-1 r + s sqrt(D^-1) NN(.) on the current
// r (c->nr), with s taken from s_ptr; optional FCG partials (z^T q, z^T r)
void nn_apply(mpml_ctx_s* c, const double* s_ptr, const float* q, double* part) {
  NNBufs b = nn_bufs(c);
  const unsigned nb = (unsigned)c->nb;
  k_nn_input<<<nb, BV, 0, c->s>>>((const float*)c->nr.p, (const float*)c->ndinv.p, s_ptr, b.x);
  nn_forward(c);
  k_nn_combine<<<nb, BV, 0, c->s>>>((const float*)c->nr.p, (const float*)c->ndinv.p, b.y, q, s_ptr, (float*)c->nz.p,
                                    part);
  c->launches += 2;
}

// gradient of the loss w.r.t. the weights for one sample, accumulated
// (scaled) into b.grad.  gy (fp32, node layout [brick][3][512]) is the loss
// gradient w.r.t. the network output; its bf16 copy is formed here.
__global__ void __launch_bounds__(512) k_nn_gout(const float* __restrict__ gy, const uint8_t* __restrict__ nflag,
                                                 __nv_bfloat16* g) {
  const int id = blockIdx.x, l = threadIdx.x;
  const uint8_t f = nflag[(int64_t)id * BV + l];
  const bool fre = (f & NF_DOF) && !(f & NF_FIXED);
  __align__(16) __nv_bfloat16 v[NNC];
#pragma unroll
  for (int ch = 0; ch < NNC; ++ch) v[ch] = __float2bfloat16_rn(0.f);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) v[ch] = __float2bfloat16_rn(fre ? gy[((int64_t)id * 3 + ch) * BV + l] : 0.f);
  uint4* dst = reinterpret_cast<uint4*>(g + ((int64_t)id * BV + l) * NNC);
  dst[0] = reinterpret_cast<const uint4*>(v)[0];
  dst[1] = reinterpret_cast<const uint4*>(v)[1];
}

void nn_backward(mpml_ctx_s* c, const float* gy, float scale) {
  set_conv_attrs();
  NNBufs b = nn_bufs(c);
  const unsigned nb = (unsigned)c->nb;
  const size_t smem = HALO_BYTES + W_BYTES, smem_w = HALO_BYTES + BV * 32;
  const uint8_t* nf = (const uint8_t*)c->nflag.p;
  const int* nbr = (const int*)c->nbr.p;
  const unsigned rb = div_up(NN_LAYER, 256);
  k_nn_gout<<<nb, BV, 0, c->s>>>(gy, nf, b.g);
  // layer 3: dW3 from (h2, g3); g_h2 = conv^T(g3) masked by h2 > 0
  k_conv_wgrad<<<nb, 256, smem_w, c->s>>>(b.h2, b.g, nbr, b.part);
  k_wgrad_reduce<<<rb, 256, 0, c->s>>>(b.part, (int)c->nb, scale, b.grad + 2 * NN_LAYER);
  k_conv<2><<<nb, 256, smem, c->s>>>(b.g, b.wb + 2 * NN_LAYER, nbr, nf, b.h2, b.g2, nullptr);
  // layer 2
  k_conv_wgrad<<<nb, 256, smem_w, c->s>>>(b.h1, b.g2, nbr, b.part);
  k_wgrad_reduce<<<rb, 256, 0, c->s>>>(b.part, (int)c->nb, scale, b.grad + NN_LAYER);
  k_conv<2><<<nb, 256, smem, c->s>>>(b.g2, b.wb + NN_LAYER, nbr, nf, b.h1, b.g, nullptr);
  // layer 1
  k_conv_wgrad<<<nb, 256, smem_w, c->s>>>(b.x, b.g, nbr, b.part);
  k_wgrad_reduce<<<rb, 256, 0, c->s>>>(b.part, (int)c->nb, scale, b.grad);
  c->launches += 9;
}

// Adam on the master weights (padded entries stay zero: their gradient is 0)
__global__ void k_adam(float* w, float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float ge = g[e];
  const float me = b1 * m[e] + (1.f - b1) * ge, ve = b2 * v[e] + (1.f - b2) * ge * ge;
  m[e] = me;
  v[e] = ve;
  w[e] -= lr * (me / c1) / (sqrtf(ve / c2) + eps);
  g[e] = 0.f;
}

void nn_adam(mpml_ctx_s* c, float lr, int step) {
  NNBufs b = nn_bufs(c);
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<div_up(3 * NN_LAYER, 256), 256, 0, c->s>>>(b.master, b.grad, b.adam_m, b.adam_v, 3 * NN_LAYER, lr, b1, b2,
                                                      1e-8f, c1, c2);
  c->launches++;
}

// weights in the oracle layout (27, Cout, Cin) per layer <-> padded master
int nn_set_weights(mpml_ctx_s* c, const float* w) {
  int rc = nn_ensure(c);
  if (rc) return rc;
  std::vector<float> pad((size_t)3 * NN_LAYER, 0.f);
  size_t off = 0;
  for (int l = 0; l < 3; ++l)
    for (int t = 0; t < 27; ++t)
      for (int n = 0; n < nn_cout(l); ++n)
        for (int k = 0; k < nn_cin(l); ++k) pad[(size_t)l * NN_LAYER + (t * NNC + n) * NNC + k] = w[off++];
  NNBufs b = nn_bufs(c);
  cudaMemcpyAsync(b.master, pad.data(), sizeof(float) * pad.size(), cudaMemcpyHostToDevice, c->s);
  cudaMemsetAsync(b.grad, 0, sizeof(float) * 3 * 3 * NN_LAYER, c->s);  // grad, adam m, adam v
  if ((rc = nn_refresh_weights(c))) return rc;
  return cuda_status(cudaStreamSynchronize(c->s));
}

int nn_get_weights(mpml_ctx_s* c, float* w, int grad) {
  if (!c->nnw.p) return MPML_ERR_ARG;
  std::vector<float> pad((size_t)3 * NN_LAYER);
  NNBufs b = nn_bufs(c);
  cudaMemcpyAsync(pad.data(), grad ? b.grad : b.master, sizeof(float) * pad.size(), cudaMemcpyDeviceToHost, c->s);
  int rc = cuda_status(cudaStreamSynchronize(c->s));
  if (rc) return rc;
  size_t off = 0;
  for (int l = 0; l < 3; ++l)
    for (int t = 0; t < 27; ++t)
      for (int n = 0; n < nn_cout(l); ++n)
        for (int k = 0; k < nn_cin(l); ++k) w[off++] = pad[(size_t)l * NN_LAYER + (t * NNC + n) * NNC + k];
  return MPML_OK;
}

int nn_weight_count() { return 27 * (3 * 16 + 16 * 16 + 16 * 3); }

float* nn_output(mpml_ctx_s* c) { return (float*)c->nny.p; }

}  // namespace mpml
