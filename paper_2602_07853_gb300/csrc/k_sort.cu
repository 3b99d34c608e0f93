// Algorithm 2, first half: binning of particles to their base centre, the
// brick set, the stable brick-major sort, active cells and DOF nodes.
//
// Base centre (Sec. 3.1, trilinear w_cp over the 8 surrounding centres):
//   s_a = x_a * inv_dx - 1/2 (double, no FMA), b_a = floor(s_a), f_a = s_a - b_a.
// Active cell: some particle has w_cp > 0, i.e. per axis c_a = b_a, or
// c_a = b_a + 1 with f_a > 0 (Algorithm 2, cells with m_c != 0).
// DOF nodes: the 8 corners of active cells.
// Sort: stable by key of the base centre = counting sort by key followed by
// ordering each key's segment by the previous particle index.
#include "mpml_internal.cuh"

namespace mpml {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? MPML_OK : MPML_ERR_CUDA; }

int ensure(Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return MPML_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  size_t want = bytes + bytes / 4;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      return MPML_ERR_NOMEM;
    }
    want = bytes;
  }
  b.bytes = want;
  return MPML_OK;
}

void free_buf(Buf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// ---------------------------------------------------------------------------
struct GridInfo {
  int n[3];
  int NB[3];
  double inv_dx;
};

__device__ __forceinline__ bool base_cell(const GridInfo& g, const double xa[3], int b[3], double f[3],
                                          int* status) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!isfinite(xa[a])) {
      atomicOr(status, ST_NONFINITE);
      return false;
    }
    double sa = __dsub_rn(__dmul_rn(xa[a], g.inv_dx), 0.5);
    double fl = floor(sa);
    if (fl < 0.0 || fl + 1.0 > (double)(g.n[a] - 1)) {
      atomicOr(status, ST_OUT_OF_DOMAIN);
      return false;
    }
    b[a] = (int)fl;
    f[a] = __dsub_rn(sa, fl);
  }
  return true;
}

__device__ __forceinline__ int64_t dense_brick(const GridInfo& g, int bx, int by, int bz) {
  return ((int64_t)bz * g.NB[1] + by) * g.NB[0] + bx;
}

template <typename T>
__global__ void k_bin_mark(int64_t np, const T* __restrict__ x, GridInfo g, uint8_t* bflag_c,
                           uint8_t* bflag_n, int* status) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double xa[3] = {(double)x[3 * p], (double)x[3 * p + 1], (double)x[3 * p + 2]};
  int b[3];
  double f[3];
  if (!base_cell(g, xa, b, f, status)) return;
  int hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) hi[a] = b[a] + (f[a] > 0.0 ? 1 : 0);
  // bricks of the active cells b..hi
  for (int bz = b[2] >> 3; bz <= hi[2] >> 3; ++bz)
    for (int by = b[1] >> 3; by <= hi[1] >> 3; ++by)
      for (int bx = b[0] >> 3; bx <= hi[0] >> 3; ++bx) bflag_c[dense_brick(g, bx, by, bz)] = 1;
  // bricks of their corner nodes b..hi+1
  for (int bz = b[2] >> 3; bz <= (hi[2] + 1) >> 3; ++bz)
    for (int by = b[1] >> 3; by <= (hi[1] + 1) >> 3; ++by)
      for (int bx = b[0] >> 3; bx <= (hi[0] + 1) >> 3; ++bx) bflag_n[dense_brick(g, bx, by, bz)] = 1;
}

// Single-block ordered compaction of the dense brick flags.
__global__ void k_compact_bricks(int64_t NBT, const uint8_t* bflag_c, const uint8_t* bflag_n, int* bmap,
                                 int* blist, int* cblist, int* nolist, int* counts) {
  __shared__ int warp_tot[3][32];
  __shared__ int carry[3];
  if (threadIdx.x == 0) carry[0] = carry[1] = carry[2] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t base = 0; base < NBT; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int fc = 0, fa = 0;
    if (i < NBT) {
      fc = bflag_c[i] ? 1 : 0;
      fa = (fc || bflag_n[i]) ? 1 : 0;
    }
    const int fo = fa && !fc;  // bricks holding DOF nodes but no active cell
    unsigned ma = __ballot_sync(0xffffffffu, fa), mc = __ballot_sync(0xffffffffu, fc),
             mo = __ballot_sync(0xffffffffu, fo);
    int pa = __popc(ma & ((1u << lane) - 1)), pc = __popc(mc & ((1u << lane) - 1)),
        po = __popc(mo & ((1u << lane) - 1));
    if (lane == 0) {
      warp_tot[0][wid] = __popc(ma);
      warp_tot[1][wid] = __popc(mc);
      warp_tot[2][wid] = __popc(mo);
    }
    __syncthreads();
    int offa = carry[0], offc = carry[1], offo = carry[2];
    for (int w = 0; w < wid; ++w) {
      offa += warp_tot[0][w];
      offc += warp_tot[1][w];
      offo += warp_tot[2][w];
    }
    if (i < NBT) {
      if (fa) {
        int id = offa + pa;
        bmap[i] = id;
        blist[id] = (int)i;
        if (fc) cblist[offc + pc] = id;
        if (fo) nolist[offo + po] = id;
      } else {
        bmap[i] = -1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 0; w < nw; ++w) {
        carry[0] += warp_tot[0][w];
        carry[1] += warp_tot[1][w];
        carry[2] += warp_tot[2][w];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    counts[0] = carry[0];
    counts[1] = carry[1];
    counts[2] = carry[2];
  }
}

__global__ void k_neighbors(int nb, const int* blist, const int* bmap, GridInfo g, int* nbr) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nb * NBR) return;
  int bi = id / NBR, j = id % NBR;
  int dxo = j % 3 - 1, dyo = (j / 3) % 3 - 1, dzo = j / 9 - 1;
  int64_t d = blist[bi];
  int bx = (int)(d % g.NB[0]), by = (int)((d / g.NB[0]) % g.NB[1]), bz = (int)(d / ((int64_t)g.NB[0] * g.NB[1]));
  int x = bx + dxo, y = by + dyo, z = bz + dzo;
  int r = -1;
  if (x >= 0 && y >= 0 && z >= 0 && x < g.NB[0] && y < g.NB[1] && z < g.NB[2]) r = bmap[dense_brick(g, x, y, z)];
  nbr[id] = r;
}

// key = compact brick of the base centre * 512 + local index; counting-sort
// rank by atomics; active-cell flags in the compact layout.
template <typename T>
__global__ void k_keys(int64_t np, const T* __restrict__ x, GridInfo g, const int* bmap, int* key, int* rank,
                       int* cnt, uint8_t* cflag, int* status) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double xa[3] = {(double)x[3 * p], (double)x[3 * p + 1], (double)x[3 * p + 2]};
  int b[3];
  double f[3];
  if (!base_cell(g, xa, b, f, status)) return;
  int cb = bmap[dense_brick(g, b[0] >> 3, b[1] >> 3, b[2] >> 3)];
  int k = cb * BV + ((b[2] & 7) * 64 + (b[1] & 7) * 8 + (b[0] & 7));
  key[p] = k;
  rank[p] = atomicAdd(&cnt[k], 1);
  for (int o = 0; o < 8; ++o) {
    int oa[3] = {o & 1, (o >> 1) & 1, (o >> 2) & 1};
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (oa[a] && !(f[a] > 0.0)) ok = false;
    if (!ok) continue;
    int c[3] = {b[0] + oa[0], b[1] + oa[1], b[2] + oa[2]};
    int id = bmap[dense_brick(g, c[0] >> 3, c[1] >> 3, c[2] >> 3)];
    cflag[(int64_t)id * BV + (c[2] & 7) * 64 + (c[1] & 7) * 8 + (c[0] & 7)] = 1;
  }
}

// ---------------------------------------------------------------------------
// Exclusive scan of int32 (3 phases, 2048 elements per block).
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024, SCAN_E = 2048;

__device__ int block_excl_scan(int v, int* sh) {
  // returns exclusive prefix within the block; sh[32] scratch; sh[32] total
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sh[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  int excl = x - v + (wid > 0 ? sh[wid - 1] : 0);
  int total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  if (threadIdx.x == 0) sh[32] = total;
  __syncthreads();
  return excl;
}

__global__ void k_scan_reduce(const int* in, int64_t n, int* bsum) {
  __shared__ int sh[33];
  int64_t base = (int64_t)blockIdx.x * SCAN_E;
  int v = 0;
  for (int j = threadIdx.x; j < SCAN_E; j += blockDim.x) {
    int64_t i = base + j;
    if (i < n) v += in[i];
  }
  block_excl_scan(v, sh);
  if (threadIdx.x == 0) bsum[blockIdx.x] = sh[32];
}

__global__ void k_scan_sums(int* bsum, int nblk, int* total) {
  __shared__ int sh[33];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblk; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < nblk ? bsum[i] : 0;
    int ex = block_excl_scan(v, sh);
    if (i < nblk) bsum[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += sh[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(const int* in, int64_t n, const int* bsum, int* out) {
  __shared__ int sh[33];
  int64_t base = (int64_t)blockIdx.x * SCAN_E;
  // each thread owns 2 consecutive elements
  int64_t i0 = base + 2 * threadIdx.x;
  int a = i0 < n ? in[i0] : 0;
  int b = i0 + 1 < n ? in[i0 + 1] : 0;
  int ex = block_excl_scan(a + b, sh) + bsum[blockIdx.x];
  if (i0 < n) out[i0] = ex;
  if (i0 + 1 < n) out[i0 + 1] = ex + a;
}

// out[0..n) = exclusive scan of in, out[n] = total.  tmp holds block sums.
static int scan_exclusive(mpml_ctx_s* c, const int* in, int* out, int64_t n, Buf& tmp) {
  int nblk = (int)div_up(n, SCAN_E);
  if (nblk < 1) nblk = 1;
  int rc = ensure(tmp, sizeof(int) * (nblk + 1));
  if (rc) return rc;
  int* bsum = (int*)tmp.p;
  k_scan_reduce<<<nblk, SCAN_T, 0, c->s>>>(in, n, bsum);
  k_scan_sums<<<1, SCAN_T, 0, c->s>>>(bsum, nblk, out + n);
  k_scan_apply<<<nblk, SCAN_T, 0, c->s>>>(in, n, bsum, out);
  c->launches += 3;
  return cuda_status(cudaGetLastError());
}

__global__ void k_scatter_perm(int64_t np, const int* key, const int* rank, const int* start, int* perm) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  perm[start[key[p]] + rank[p]] = (int)p;
}

// order each key segment by previous index (insertion sort; segments are short)
__global__ void k_segsort(int64_t nkeys, const int* start, int* perm) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nkeys) return;
  int s = start[k], e = start[k + 1];
  if (e - s < 2) return;
  for (int i = s + 1; i < e; ++i) {
    int v = perm[i];
    int j = i - 1;
    while (j >= s && perm[j] > v) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = v;
  }
}

template <typename T>
__global__ void k_gather(int64_t np, const int* perm, const T* x, const T* v, const T* F, const T* G, const T* m,
                         const T* V, const int32_t* mat, T* xs, T* vs, T* Fs, T* Gs, T* ms, T* Vs, int32_t* mats,
                         int* keys_sorted, const int* keys, int32_t* perm_out, int nm, int* status) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np) return;
  int64_t p = perm[s];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xs[3 * s + a] = x[3 * p + a];
    vs[3 * s + a] = v[3 * p + a];
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    Fs[9 * s + a] = F[9 * p + a];
    Gs[9 * s + a] = G[9 * p + a];
  }
  ms[s] = m[p];
  Vs[s] = V[p];
  int32_t k = mat[p];
  if (k < 0 || k >= nm) atomicOr(status, ST_BADMAT);
  mats[s] = k;
  keys_sorted[s] = keys[p];
  if (perm_out) perm_out[s] = (int32_t)p;
}

// DOF node flags: corners of active cells (cell-brick CTAs, 512 threads)
__global__ void k_mark_nodes(const int* cblist, const int* nbr, const uint8_t* cflag, uint8_t* nflag) {
  int id = cblist[blockIdx.x];
  int l = threadIdx.x;
  if (!cflag[(int64_t)id * BV + l]) return;
  int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
  for (int o = 0; o < 8; ++o) {
    int x = lx + (o & 1), y = ly + ((o >> 1) & 1), z = lz + ((o >> 2) & 1);
    int bx = x >> 3, by = y >> 3, bz = z >> 3;
    int t = nbr[id * NBR + nbr_index(bx, by, bz)];
    if (t >= 0) nflag[(int64_t)t * BV + (z & 7) * 64 + (y & 7) * 8 + (x & 7)] = NF_DOF;
  }
}

struct BoundaryInfo {
  int n[3];
  int wall;
  int has_plate;
  double dx, t;
  double lo[3], hi[3], vel[3];
};

// Dirichlet rule: sticky outer wall layers, then the moving box.
__global__ void k_node_setup(const int* blist, GridInfo g, BoundaryInfo bi, uint8_t* nflag, double* vfix) {
  int id = blockIdx.x;
  int l = threadIdx.x;
  int64_t slot = (int64_t)id * BV + l;
  uint8_t f = nflag[slot];
  double* vf = vfix + (int64_t)id * 3 * BV + l;
  vf[0] = vf[BV] = vf[2 * BV] = 0.0;
  if (!(f & NF_DOF)) return;
  int64_t d = blist[id];
  int bx = (int)(d % g.NB[0]), by = (int)((d / g.NB[0]) % g.NB[1]), bz = (int)(d / ((int64_t)g.NB[0] * g.NB[1]));
  int ijk[3] = {bx * 8 + (l & 7), by * 8 + ((l >> 3) & 7), bz * 8 + (l >> 6)};
  bool fixed = false;
  for (int a = 0; a < 3; ++a)
    if (ijk[a] < bi.wall || ijk[a] > bi.n[a] - bi.wall) fixed = true;
  if (!fixed && bi.has_plate) {
    bool in = true;
    for (int a = 0; a < 3; ++a) {
      double xa = __dmul_rn((double)ijk[a], bi.dx);
      double sh = __dmul_rn(bi.vel[a], bi.t);
      double lo = __dadd_rn(bi.lo[a], sh), hi = __dadd_rn(bi.hi[a], sh);
      if (!(xa >= lo && xa <= hi)) in = false;
    }
    if (in) {
      fixed = true;
      vf[0] = bi.vel[0];
      vf[BV] = bi.vel[1];
      vf[2 * BV] = bi.vel[2];
    }
  }
  if (fixed) nflag[slot] = f | NF_FIXED;
}

static GridInfo grid_info(mpml_ctx_s* c) {
  GridInfo g;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = c->d.n[a];
    g.NB[a] = c->NB[a];
  }
  g.inv_dx = c->d.inv_dx;
  return g;
}

// First half of the resample: brick flags and their compaction, with the
// counts copied to the host (asynchronously; the caller synchronises).
template <typename T>
static int resample_begin_t(mpml_ctx_s* c, const void* x_) {
  const T* x = (const T*)x_;
  const int64_t np = c->np_count;
  GridInfo g = grid_info(c);
  int rc;
  int* status = (int*)c->status.p;
  cudaStream_t s = c->s;
  // brick flags
  if ((rc = ensure(c->bflag_c, c->NBT)) || (rc = ensure(c->bflag_n, c->NBT)) ||
      (rc = ensure(c->bmap, sizeof(int) * c->NBT)) || (rc = ensure(c->blist, sizeof(int) * c->NBT)) ||
      (rc = ensure(c->cblist, sizeof(int) * c->NBT)) || (rc = ensure(c->nolist, sizeof(int) * c->NBT)))
    return rc;
  cudaMemsetAsync(c->bflag_c.p, 0, c->NBT, s);
  cudaMemsetAsync(c->bflag_n.p, 0, c->NBT, s);
  if (np > 0) {
    k_bin_mark<T><<<div_up(np, 256), 256, 0, s>>>(np, x, g, (uint8_t*)c->bflag_c.p, (uint8_t*)c->bflag_n.p, status);
    c->launches++;
  }
  k_compact_bricks<<<1, 1024, 0, s>>>(c->NBT, (const uint8_t*)c->bflag_c.p, (const uint8_t*)c->bflag_n.p,
                                      (int*)c->bmap.p, (int*)c->blist.p, (int*)c->cblist.p, (int*)c->nolist.p,
                                      (int*)&((DevScalars*)c->scal.p)->counter[5]);
  c->launches++;
  // counts (and the status word) to the host: one synchronisation per resample
  cudaMemcpyAsync(c->hscal, c->scal.p, sizeof(DevScalars), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(c->hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  return cuda_status(cudaGetLastError());
}

// Second half, after the counts arrived: neighbours, keys, counting sort,
// gather, DOF nodes and the Dirichlet set.
template <typename T>
static int resample_end_t(mpml_ctx_s* c, const void* x_, const void* v_, const void* F_, const void* G_,
                          const void* m_, const void* V_, const int32_t* mat, int32_t* perm_out) {
  const T* x = (const T*)x_;
  const int64_t np = c->np_count;
  GridInfo g = grid_info(c);
  int rc;
  int* status = (int*)c->status.p;
  cudaStream_t s = c->s;
  if (*c->hstatus & ST_NONFINITE) return MPML_ERR_NONFINITE;
  if (*c->hstatus & ST_OUT_OF_DOMAIN) return MPML_ERR_OUT_OF_DOMAIN;
  c->nb = c->hscal->counter[5];
  c->ncb = c->hscal->counter[6];
  c->nnob = c->hscal->counter[7];
  const int64_t nb = c->nb, nslots = nb * BV;
  // neighbour table
  if ((rc = ensure(c->nbr, sizeof(int) * NBR * (nb ? nb : 1)))) return rc;
  if (nb > 0) {
    k_neighbors<<<div_up(nb * NBR, 256), 256, 0, s>>>((int)nb, (const int*)c->blist.p, (const int*)c->bmap.p, g,
                                                       (int*)c->nbr.p);
    c->launches++;
  }
  // particle keys and counting sort
  if ((rc = ensure(c->pkey, sizeof(int) * np)) || (rc = ensure(c->prank, sizeof(int) * np)) ||
      (rc = ensure(c->pperm, sizeof(int) * np)) || (rc = ensure(c->pbase, sizeof(int) * np)) ||
      (rc = ensure(c->cnt, sizeof(int) * (nslots + 1))) || (rc = ensure(c->start, sizeof(int) * (nslots + 1))) ||
      (rc = ensure(c->cflag, nslots)) || (rc = ensure(c->nflag, nslots)))
    return rc;
  cudaMemsetAsync(c->cnt.p, 0, sizeof(int) * (nslots + 1), s);
  cudaMemsetAsync(c->cflag.p, 0, nslots ? nslots : 1, s);
  cudaMemsetAsync(c->nflag.p, 0, nslots ? nslots : 1, s);
  if (np > 0) {
    k_keys<T><<<div_up(np, 256), 256, 0, s>>>(np, x, g, (const int*)c->bmap.p, (int*)c->pbase.p, (int*)c->prank.p,
                                              (int*)c->cnt.p, (uint8_t*)c->cflag.p, status);
    c->launches++;
  }
  if ((rc = scan_exclusive(c, (const int*)c->cnt.p, (int*)c->start.p, nslots, c->scan_tmp))) return rc;
  const size_t es = sizeof(T);
  if ((rc = ensure(c->px, es * 3 * np)) || (rc = ensure(c->pv, es * 3 * np)) || (rc = ensure(c->pF, es * 9 * np)) ||
      (rc = ensure(c->pG, es * 9 * np)) || (rc = ensure(c->pm, es * np)) || (rc = ensure(c->pV, es * np)) ||
      (rc = ensure(c->pmat, sizeof(int32_t) * np)))
    return rc;
  if (np > 0) {
    k_scatter_perm<<<div_up(np, 256), 256, 0, s>>>(np, (const int*)c->pbase.p, (const int*)c->prank.p,
                                                   (const int*)c->start.p, (int*)c->pperm.p);
    k_segsort<<<div_up(nslots, 256), 256, 0, s>>>(nslots, (const int*)c->start.p, (int*)c->pperm.p);
    k_gather<T><<<div_up(np, 256), 256, 0, s>>>(
        np, (const int*)c->pperm.p, x, (const T*)v_, (const T*)F_, (const T*)G_, (const T*)m_, (const T*)V_, mat,
        (T*)c->px.p, (T*)c->pv.p, (T*)c->pF.p, (T*)c->pG.p, (T*)c->pm.p, (T*)c->pV.p, (int32_t*)c->pmat.p,
        (int*)c->pkey.p, (const int*)c->pbase.p, perm_out, c->nm, status);
    c->launches += 3;
  }
  // DOF nodes and Dirichlet set
  if (c->ncb > 0) {
    k_mark_nodes<<<(unsigned)c->ncb, BV, 0, s>>>((const int*)c->cblist.p, (const int*)c->nbr.p,
                                                 (const uint8_t*)c->cflag.p, (uint8_t*)c->nflag.p);
    c->launches++;
  }
  if ((rc = ensure(c->nvfix, sizeof(double) * 3 * nslots))) return rc;
  BoundaryInfo bi;
  for (int a = 0; a < 3; ++a) {
    bi.n[a] = c->d.n[a];
    bi.lo[a] = c->d.plate_lo[a];
    bi.hi[a] = c->d.plate_hi[a];
    bi.vel[a] = c->d.plate_vel[a];
  }
  bi.wall = c->d.wall_layers;
  bi.has_plate = c->d.has_plate;
  bi.dx = c->d.dx;
  bi.t = c->time;
  if (nb > 0) {
    k_node_setup<<<(unsigned)nb, BV, 0, s>>>((const int*)c->blist.p, g, bi, (uint8_t*)c->nflag.p, (double*)c->nvfix.p);
    c->launches++;
  }
  return cuda_status(cudaGetLastError());
}

int resample_device_begin(mpml_ctx_s* c, const void* x) {
  return c->fp64 ? resample_begin_t<double>(c, x) : resample_begin_t<float>(c, x);
}

int resample_device_end(mpml_ctx_s* c, const void* x, const void* v, const void* F, const void* G, const void* m,
                        const void* V, const int32_t* mat, int32_t* perm_out) {
  if (c->fp64) return resample_end_t<double>(c, x, v, F, G, m, V, mat, perm_out);
  return resample_end_t<float>(c, x, v, F, G, m, V, mat, perm_out);
}

int resample_device(mpml_ctx_s* c, const void* x, const void* v, const void* F, const void* G, const void* m,
                    const void* V, const int32_t* mat, int32_t* perm_out) {
  int rc = resample_device_begin(c, x);
  if (rc) return rc;
  if ((rc = cuda_status(cudaStreamSynchronize(c->s)))) return rc;
  return resample_device_end(c, x, v, F, G, m, V, mat, perm_out);
}

}  // namespace mpml
