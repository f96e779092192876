// H-matrix far field: a fast application of the 4-point-rule far-field part A4 of the system
// operator (the role the paper gives a fast multipole method, Sec. 2.1, the paragraph on the
// fast solver).  Hierarchical matrices (Hackbusch 1999) with adaptive cross approximation
// (Bebendorf 2000, "Approximation of boundary element matrices", Numer. Math. 86):
//   * the cluster tree and block partition are host index work (hmatrix_tree.cpp);
//   * aca_kernel: one CTA per (low-rank block, frequency) runs the partially pivoted cross
//     approximation of the block's 3 m x 3 n matrix with three row classes (the vector
//     components; trial steps from each class before it stops), entries of A4 evaluated on the
//     fly in FP32 with float-float source-target distances, factors written to a scratch area;
//   * copy_factors_kernel: moves each block's U (3 m x k) and V (3 n x k) into exactly sized
//     storage, undoing the column scaling of displacement-given columns;
//   * lowrank_apply_kernel: one CTA per (group of up to 4 low-rank blocks of one target cluster,
//     frequency): per block t = V^T x_sigma (a warp per rank), y_tau += U t, then one FP64
//     atomic add per output into the far-field accumulator;
//   * dense_apply_kernel: one CTA per (group of up to 4 dense source leaves of one target leaf,
//     frequency): summed on the fly with the 4-point rule, own element excluded.
// The near-field and own-element corrections of the FP32 operator then run unchanged.  The
// low-rank apply reads each factor once per application (HBM-bound); the dense part is bound by
// the FP32 kernel arithmetic like the direct far kernel.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "kernel_math.cuh"

namespace bem {

constexpr int kHMaxRank = 256;   // bound of max_rank (shared-memory arrays of the kernels)
constexpr int kAcaThreads = 128;
constexpr int kApplyThreads = 256;
constexpr int kDenseThreads = 128;
constexpr int64_t kGroupBlocks = 4;  // blocks (low-rank) or source leaves (dense) per apply CTA

struct HGeo {
  const float4* q4;    // [ne][4] (x, y, z, w * area)
  const float4* q4lo;  // low parts of the points
  const float4* cen;   // [ne] centroid
  const float4* cenlo;
  const float4* nrm;   // [ne] unit normal
  const int8_t* bc;    // [ne] or null (all traction-given)
  const int32_t* perm; // tree position -> element
  MatC<float> m;
  float cscale;        // mu / D: displacement-given columns inside the cross approximation
};

// B[3c + d] = sum_q w_q K_e(x_t, y_q)_cd, the A4 block of target element t and source element e
// (K_e = T for a traction-given e, -U for a displacement-given one), zero for t == e; `scaled`
// multiplies displacement-given columns by g.cscale.
__device__ __forceinline__ void pair_block(const HGeo& g, int t, int e, const FreqC<float>& fc, bool scaled,
                                           cx<float>* B) {
#pragma unroll
  for (int k = 0; k < 9; ++k) B[k] = mk(0.f, 0.f);
  if (t == e) return;
  const float4 c = g.cen[t], cl = g.cenlo[t], n = g.nrm[e];
  const bool useU = g.bc && g.bc[e] == BEM_BC_DISPLACEMENT;
  const float nv[3] = {n.x, n.y, n.z};
#pragma unroll 1
  for (int q = 0; q < 4; ++q) {
    const float4 p = g.q4[4 * e + q], pl = g.q4lo[4 * e + q];
    const Dist<float> D = distance(p.x, p.y, p.z, pl, c.x, c.y, c.z, cl, false);
    const float inv_r2 = D.rinv * D.rinv;
    const float rh[3] = {D.dx * D.rinv, D.dy * D.rinv, D.dz * D.rinv};
    const Radial<float> K = radial(D.r, inv_r2, fc, g.m, D.r_lo);
    if (!useU) {
      const float drdn = rh[0] * nv[0] + rh[1] * nv[1] + rh[2] * nv[2];
      const float cw = p.w * inv_r2 * (float)kInv4Pi;
      const TCoef<float> T = tcoef(K, g.m);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float diag = a == d ? drdn : 0.f;
          const cx<float> v = (diag + nv[a] * rh[d]) * T.A + rh[a] * (nv[d] * T.q1 + (drdn * rh[d]) * T.q2);
          B[3 * a + d] = B[3 * a + d] + cw * v;
        }
    } else {
      const float cu = p.w * D.rinv * g.m.inv4pimu;
      const cx<float> psi = K.Es - K.J;
      const cx<float> chi = axpy(-3.f, K.J, K.P);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const cx<float> v = (a == d ? psi : mk(0.f, 0.f)) - (rh[a] * rh[d]) * chi;
          B[3 * a + d] = B[3 * a + d] + cu * v;
        }
    }
  }
  if (useU) {
    const float sgn = scaled ? -g.cscale : -1.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) B[k] = sgn * B[k];
  }
}

__device__ __forceinline__ float abs2(cx<float> z) { return z.r * z.r + z.i * z.i; }

// ------------------------------------------------------------------------------- reductions
// Block-wide argmax of (v, i) with the smallest index on ties; v < 0 marks "no candidate".
// Every thread receives the result.  Uses sv/si (one slot per warp) and a trailing barrier.
__device__ __forceinline__ void block_argmax(float v, int i, float* sv, int* si, float& bv, int& bi) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_down_sync(0xffffffffu, v, o);
    const int oi = __shfl_down_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
  __syncthreads();
  if (lane == 0) {
    sv[w] = v;
    si[w] = i;
  }
  __syncthreads();
  bv = sv[0];
  bi = si[0];
  for (int k = 1; k < nw; ++k)
    if (sv[k] > bv || (sv[k] == bv && si[k] < bi)) {
      bv = sv[k];
      bi = si[k];
    }
  __syncthreads();
}

__device__ __forceinline__ float block_sum(float v, float* sv) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sv[w] = v;
  __syncthreads();
  float s = 0.f;
  for (int k = 0; k < nw; ++k) s += sv[k];
  __syncthreads();
  return s;
}

__device__ __forceinline__ cx<float> warp_sum(cx<float> z) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    z.r += __shfl_down_sync(0xffffffffu, z.r, o);
    z.i += __shfl_down_sync(0xffffffffu, z.i, o);
  }
  return z;
}

}  // namespace bem

namespace bem {

// ------------------------------------------------------------------------------- ACA
struct AcaItem {
  int32_t blk, f;  // low-rank block, frequency
  int64_t off;     // float2 offset of the item's scratch: U [kmax][3 tn], then V [kmax][3 sn]
};

struct AcaArgs {
  HGeo g;
  const int4* lr;          // (t0, tn, s0, sn)
  const FreqC<float>* fc;  // [F]
  const AcaItem* items;
  float2* scratch;
  int32_t* rank;           // [items]
  int32_t* capped;         // counter of items that ended at kmax
  int kmax;
  int nmax;                // 3 * the largest block side: shared-memory stride
  float eps2;              // eps^2
};

// Partially pivoted cross approximation of one (block, frequency) item, rows in three classes
// (row i = 3 * target + component, class i % 3).  Step k: the residual of pivot row i (entries
// minus the current approximation) picks the pivot column j of largest modulus (first on ties);
// v = residual row / pivot entry, u = residual column j; the squared Frobenius norm of the
// approximation would grow by 2 Re sum_{l<k} <u_l, u><v_l, v> + |u|^2 |v|^2, and the step is
// small when |u| |v| <= eps |S|.  A step that is not small is appended and the next pivot row is
// the unused row of largest |u|; a small step is not appended (below the tolerance; after an
// exact approximation its pivot is rounding noise), and a trial row from each class follows in
// turn (the unused row of that class with the largest |u| of the last step); the approximation
// ends when every trial is small.  A residual row that vanishes counts as small, except before
// the first update, where the next unused row is taken.  Every iteration marks one row as used,
// so the loop ends after at most 3 tn iterations.
__global__ void __launch_bounds__(kAcaThreads) aca_kernel(const AcaArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* row = reinterpret_cast<cx<float>*>(smem_raw);           // [nmax] residual row, then v
  cx<float>* ucol = row + a.nmax;                                     // [nmax] last u
  unsigned char* used = reinterpret_cast<unsigned char*>(ucol + a.nmax);  // [nmax]
  __shared__ cx<float> coef[kHMaxRank];
  __shared__ cx<float> du[kHMaxRank], dv[kHMaxRank];
  __shared__ float sv[kAcaThreads / 32];
  __shared__ int si[kAcaThreads / 32];
  __shared__ float s_norm2;
  __shared__ int s_k, s_i, s_trial, s_small, s_have, s_done;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const AcaItem it = a.items[blockIdx.x];
  const int4 B = a.lr[it.blk];
  const int t0 = B.x, tn = B.y, s0 = B.z, sn = B.w;
  const int M = 3 * tn, N = 3 * sn;
  float2* U = a.scratch + it.off;
  float2* V = U + (int64_t)a.kmax * M;
  const FreqC<float> fc = a.fc[it.f];
  for (int i = tid; i < M; i += kAcaThreads) used[i] = 0;
  if (tid == 0) {
    s_norm2 = 0.f;
    s_k = 0;
    s_i = 0;
    s_trial = -1;
    s_have = 0;
    s_done = 0;
  }
  __syncthreads();

  for (int iter = 0; iter < M; ++iter) {
    const int k = s_k, i = s_i;
    if (k >= a.kmax) break;
    // ---- residual of pivot row i
    for (int l = tid; l < k; l += kAcaThreads) {
      const float2 u = U[(int64_t)l * M + i];
      coef[l] = mk(u.x, u.y);
    }
    __syncthreads();
    {
      const int te = a.g.perm[t0 + i / 3], c = i % 3;
      for (int el = tid; el < sn; el += kAcaThreads) {
        cx<float> B9[9];
        pair_block(a.g, te, a.g.perm[s0 + el], fc, true, B9);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int j = 3 * el + d;
          cx<float> v = B9[3 * c + d];
          for (int l = 0; l < k; ++l) {
            const float2 w = V[(int64_t)l * N + j];
            v = v - coef[l] * mk(w.x, w.y);
          }
          row[j] = v;
        }
      }
    }
    if (tid == 0) used[i] = 1;
    __syncthreads();
    float bv = -1.f;
    int bj = 0x7fffffff;
    for (int j = tid; j < N; j += kAcaThreads) {
      const float m2 = abs2(row[j]);
      if (m2 > bv) {
        bv = m2;
        bj = j;
      }
    }
    float amax;
    int jstar;
    block_argmax(bv, bj, sv, si, amax, jstar);
    bool small;
    if (amax == 0.f) {
      small = true;
      if (k == 0 && s_trial < 0) {
        // a vanishing first row: the next unused row in index order
        float cv = -1.f;
        int ci = 0x7fffffff;
        for (int r = tid; r < M; r += kAcaThreads)
          if (!used[r] && ci == 0x7fffffff) {
            cv = 0.f;
            ci = r;
          }
        float rv;
        int ri;
        block_argmax(cv, ci, sv, si, rv, ri);
        if (tid == 0) {
          if (rv < 0.f) s_done = 2;
          else s_i = ri;
        }
        __syncthreads();
        if (s_done) break;
        continue;
      }
    } else {
      // ---- v = residual row / pivot, u = residual column
      const cx<float> piv = row[jstar];
      const float inv2 = 1.f / abs2(piv);
      const cx<float> inv = mk(piv.r * inv2, -piv.i * inv2);
      __syncthreads();   // every thread has read row[jstar]
      for (int j = tid; j < N; j += kAcaThreads) {
        const cx<float> v = row[j] * inv;
        row[j] = v;
        V[(int64_t)k * N + j] = make_float2(v.r, v.i);
      }
      for (int l = tid; l < k; l += kAcaThreads) {
        const float2 w = V[(int64_t)l * N + jstar];
        coef[l] = mk(w.x, w.y);
      }
      __syncthreads();
      {
        const int se = a.g.perm[s0 + jstar / 3], d = jstar % 3;
        for (int el = tid; el < tn; el += kAcaThreads) {
          cx<float> B9[9];
          pair_block(a.g, a.g.perm[t0 + el], se, fc, true, B9);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int r = 3 * el + c;
            cx<float> u = B9[3 * c + d];
            for (int l = 0; l < k; ++l) {
              const float2 w = U[(int64_t)l * M + r];
              u = u - coef[l] * mk(w.x, w.y);
            }
            ucol[r] = u;
            U[(int64_t)k * M + r] = make_float2(u.r, u.i);
          }
        }
      }
      __syncthreads();
      // ---- norms: |u|^2, |v|^2 and <u_l, u>, <v_l, v> for l < k
      float nu = 0.f, nv = 0.f;
      for (int r = tid; r < M; r += kAcaThreads) nu += abs2(ucol[r]);
      for (int j = tid; j < N; j += kAcaThreads) nv += abs2(row[j]);
      nu = block_sum(nu, sv);
      nv = block_sum(nv, sv);
      for (int l = warp; l < k; l += kAcaThreads / 32) {
        cx<float> su = mk(0.f, 0.f), sw = mk(0.f, 0.f);
        for (int r = lane; r < M; r += 32) {
          const float2 w = U[(int64_t)l * M + r];
          su = su + conj(mk(w.x, w.y)) * ucol[r];
        }
        for (int j = lane; j < N; j += 32) {
          const float2 w = V[(int64_t)l * N + j];
          sw = sw + conj(mk(w.x, w.y)) * row[j];
        }
        su = warp_sum(su);
        sw = warp_sum(sw);
        if (lane == 0) {
          du[l] = su;
          dv[l] = sw;
        }
      }
      __syncthreads();
      if (tid == 0) {
        float cross = 0.f;
        for (int l = 0; l < k; ++l) cross += (du[l] * dv[l]).r;
        const float grown = fmaxf(s_norm2 + 2.f * cross + nu * nv, 0.f);
        s_small = (nu * nv <= a.eps2 * grown) ? 1 : 0;
        if (!s_small) {  // appended; a small step's slot k is overwritten by the next step
          s_norm2 = grown;
          s_k = k + 1;
        }
        s_have = 1;
      }
      __syncthreads();
      small = s_small != 0;
    }
    // ---- next pivot row
    if (small) {
      int c = s_trial + 1, nxt = -1;
      for (; c < 3; ++c) {
        float cv = -1.f;
        int ci = 0x7fffffff;
        for (int r = c + 3 * tid; r < M; r += 3 * kAcaThreads) {
          if (used[r]) continue;
          const float m2 = s_have ? abs2(ucol[r]) : 0.f;
          if (m2 > cv) {
            cv = m2;
            ci = r;
          }
        }
        float rv;
        int ri;
        block_argmax(cv, ci, sv, si, rv, ri);
        if (rv >= 0.f) {
          nxt = ri;
          break;
        }
      }
      if (tid == 0) {
        if (nxt < 0) s_done = 1;
        else {
          s_trial = c;
          s_i = nxt;
        }
      }
    } else {
      float cv = -1.f;
      int ci = 0x7fffffff;
      for (int r = tid; r < M; r += kAcaThreads) {
        if (used[r]) continue;
        const float m2 = abs2(ucol[r]);
        if (m2 > cv) {
          cv = m2;
          ci = r;
        }
      }
      float rv;
      int ri;
      block_argmax(cv, ci, sv, si, rv, ri);
      if (tid == 0) {
        s_trial = -1;
        if (rv < 0.f) s_done = 2;
        else s_i = ri;
      }
    }
    __syncthreads();
    if (s_done) break;
  }
  if (tid == 0) {
    a.rank[blockIdx.x] = s_k;
    if (!s_done && s_k >= a.kmax) atomicAdd(a.capped, 1);
  }
}

// Copy each item's k columns of U and V into its final storage (U then V, contiguous), V's
// displacement-given rows divided by the column scale.
struct CopyArgs {
  const int4* lr;
  const AcaItem* items;
  const float2* scratch;
  const int32_t* rank;
  float2* const* dst;
  const int32_t* perm;
  const int8_t* bc;
  float inv_cscale;
  int kmax;
};

__global__ void copy_factors_kernel(const CopyArgs a) {
  const AcaItem it = a.items[blockIdx.x];
  const int k = a.rank[blockIdx.x];
  if (k == 0) return;
  const int4 B = a.lr[it.blk];
  const int M = 3 * B.y, N = 3 * B.w;
  const float2* U = a.scratch + it.off;
  const float2* V = U + (int64_t)a.kmax * M;
  float2* out = a.dst[blockIdx.x];
  const int64_t nu = (int64_t)k * M, nv = (int64_t)k * N;
  for (int64_t t = threadIdx.x; t < nu; t += blockDim.x) out[t] = U[t];
  for (int64_t t = threadIdx.x; t < nv; t += blockDim.x) {
    const int j = (int)(t % N);
    const int e = a.perm[B.z + j / 3];
    float2 w = V[t];
    if (a.bc && a.bc[e] == BEM_BC_DISPLACEMENT) {
      w.x *= a.inv_cscale;
      w.y *= a.inv_cscale;
    }
    out[nu + t] = w;
  }
}

// ------------------------------------------------------------------------------- apply
struct LowRankArgs {
  const int32_t* perm;
  const int4* lr;              // (t0, tn, s0, sn)
  const int4* tgrp;            // (t0, tn, first, count)
  const int32_t* tblk;
  const int32_t* rank;         // [F][n_lr]
  const float2* const* fptr;   // [F][n_lr]
  const cx<float>* x;          // [F][ne][3]
  double* yacc;                // [F][ne][6]
  const int32_t* flist;
  int64_t ne, n_lr;
  int nmax;
};

// One CTA per (group of a target cluster's low-rank blocks, listed frequency): the sum over the
// group of U (V^T x_sigma), accumulated in shared memory, then added to the FP64 far-field sums.
__global__ void __launch_bounds__(kApplyThreads) lowrank_apply_kernel(const LowRankArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* xs = reinterpret_cast<cx<float>*>(smem_raw);  // [nmax] source values
  cx<float>* ys = xs + a.nmax;                              // [nmax] target sums
  __shared__ cx<float> ts[kHMaxRank];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t f = a.flist[blockIdx.y];
  const int4 G = a.tgrp[blockIdx.x];
  const int M = 3 * G.y;
  for (int i = tid; i < M; i += kApplyThreads) ys[i] = mk(0.f, 0.f);
  for (int q = 0; q < G.w; ++q) {
    const int b = a.tblk[G.z + q];
    const int k = a.rank[f * a.n_lr + b];
    if (k == 0) continue;
    const int4 B = a.lr[b];
    const int N = 3 * B.w;
    const float2* U = a.fptr[f * a.n_lr + b];
    const float2* V = U + (int64_t)k * M;
    __syncthreads();  // the previous block's xs and ts are no longer read
    for (int j = tid; j < N; j += kApplyThreads) xs[j] = a.x[(f * a.ne + a.perm[B.z + j / 3]) * 3 + j % 3];
    __syncthreads();
    for (int l = warp; l < k; l += kApplyThreads / 32) {
      cx<float> acc = mk(0.f, 0.f);
      const float2* v = V + (int64_t)l * N;
#pragma unroll 4
      for (int j = lane; j < N; j += 32) {
        const float2 w = v[j];
        acc = cfma(mk(w.x, w.y), xs[j], acc);
      }
      acc = warp_sum(acc);
      if (lane == 0) ts[l] = acc;
    }
    __syncthreads();
    for (int i = tid; i < M; i += kApplyThreads) {
      cx<float> acc = ys[i];
#pragma unroll 4
      for (int l = 0; l < k; ++l) {
        const float2 u = U[(int64_t)l * M + i];
        acc = cfma(mk(u.x, u.y), ts[l], acc);
      }
      ys[i] = acc;
    }
  }
  __syncthreads();
  for (int i = tid; i < M; i += kApplyThreads) {
    double* yo = a.yacc + (f * a.ne + a.perm[G.x + i / 3]) * 6 + 2 * (i % 3);
    atomicAdd(yo, (double)ys[i].r);
    atomicAdd(yo + 1, (double)ys[i].i);
  }
}

struct DenseArgs {
  HGeo g;
  const int4* dgrp;            // (t0, tn, first, count)
  const int2* dsrc;            // (s0, sn)
  const FreqC<float>* fc;
  const cx<float>* x;
  double* yacc;
  const int32_t* flist;
  int64_t ne;
};

// One CTA per (group of a target leaf's dense source leaves, listed frequency): lanes over 32
// targets at a time, the four warps over interleaved source elements of the group's blocks; the
// four partial sums of a target are added in shared memory and then to the FP64 far-field sums.
__global__ void __launch_bounds__(kDenseThreads) dense_apply_kernel(const DenseArgs a) {
  __shared__ cx<float> red[kDenseThreads / 32][32][3];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t f = a.flist[blockIdx.y];
  const int4 G = a.dgrp[blockIdx.x];
  const FreqC<float> fc = a.fc[f];
  for (int i0 = 0; i0 < G.y; i0 += 32) {
    const int i = i0 + lane;
    cx<float> o[3] = {mk(0.f, 0.f), mk(0.f, 0.f), mk(0.f, 0.f)};
    if (i < G.y) {
      const int t = a.g.perm[G.x + i];
      for (int q = 0; q < G.w; ++q) {
        const int2 S = a.dsrc[G.z + q];
        for (int el = warp; el < S.y; el += kDenseThreads / 32) {
          const int e = a.g.perm[S.x + el];
          cx<float> B9[9];
          pair_block(a.g, t, e, fc, false, B9);
          const cx<float>* xe = a.x + (f * a.ne + e) * 3;
          const cx<float> x0 = xe[0], x1 = xe[1], x2 = xe[2];
#pragma unroll
          for (int c = 0; c < 3; ++c) o[c] = cfma(B9[3 * c + 2], x2, cfma(B9[3 * c + 1], x1, cfma(B9[3 * c], x0, o[c])));
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) red[warp][lane][c] = o[c];
    __syncthreads();
    if (warp == 0 && i < G.y) {
      double* yo = a.yacc + (f * a.ne + a.g.perm[G.x + i]) * 6;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cx<float> s = red[0][lane][c];
        for (int w = 1; w < kDenseThreads / 32; ++w) s = s + red[w][lane][c];
        atomicAdd(yo + 2 * c, (double)s.r);
        atomicAdd(yo + 2 * c + 1, (double)s.i);
      }
    }
    __syncthreads();
  }
}

}  // namespace bem

namespace bem {

static HGeo make_geo(bem_ctx* ctx) {
  HGeo g;
  g.q4 = ctx->mesh.q4_32.as<float4>();
  g.q4lo = ctx->mesh.q4_32lo.as<float4>();
  g.cen = ctx->mesh.c32.as<float4>();
  g.cenlo = ctx->mesh.c32lo.as<float4>();
  g.nrm = ctx->mesh.n32.as<float4>();
  g.bc = ctx->bc.set ? ctx->bc.d_type.as<int8_t>() : nullptr;
  g.perm = ctx->hm.perm.as<int32_t>();
  g.m = mat_constants32(ctx->mat);
  g.cscale = (float)(ctx->mat.mu / ctx->mesh.diam);
  return g;
}

static void check_params(const bem_hmatrix_params& p) {
  BEM_REQUIRE(p.leaf >= 1 && p.leaf <= 128, "hmatrix leaf must be in 1..128");
  BEM_REQUIRE(p.max_block >= p.leaf && p.max_block <= 1024, "hmatrix max_block must be in leaf..1024");
  BEM_REQUIRE(p.max_rank >= 1 && p.max_rank <= kHMaxRank, "hmatrix max_rank must be in 1..256");
  BEM_REQUIRE(p.eta > 0.0 && std::isfinite(p.eta), "hmatrix eta must be > 0");
  BEM_REQUIRE(p.eps > 0.0 && p.eps < 1.0, "hmatrix eps must be in (0, 1)");
  BEM_REQUIRE(p.max_freqs >= 0, "hmatrix max_freqs must be >= 0");
}

template <class T>
static void upload(bem_ctx* ctx, DevBuf& d, const std::vector<T>& h) {
  d.reserve(sizeof(T) * std::max<size_t>(h.size(), 1));
  if (!h.empty())
    BEM_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, ctx->stream));
}

// Tree, partition and the grouped block lists of the current mesh and parameters.
static void ensure_structure(bem_ctx* ctx) {
  HMat& H = ctx->hm;
  if (H.have_structure) return;
  const Mesh& me = ctx->mesh;
  const int64_t ne = me.ne, nv = (int64_t)me.verts.size() / 3;
  hm::cluster_tree(me.verts.data(), nv, me.tris.data(), ne, H.prm.leaf, H.tree);
  hm::block_partition(H.tree, H.prm.eta, H.prm.max_block, H.part);
  const hm::Tree& t = H.tree;
  const int64_t nc = t.n();
  const std::vector<int32_t>& LR = H.part.lowrank;
  const std::vector<int32_t>& DN = H.part.dense;
  H.n_lr = (int64_t)LR.size() / 2;
  H.n_dn = (int64_t)DN.size() / 2;
  std::vector<int4> lr(H.n_lr);
  H.max_lr = 1;
  H.lr_pairs = 0;
  std::vector<int64_t> cnt(nc + 1, 0);
  for (int64_t b = 0; b < H.n_lr; ++b) {
    const int32_t a = LR[2 * b], c = LR[2 * b + 1];
    lr[b] = make_int4(t.begin[a], t.size[a], t.begin[c], t.size[c]);
    H.max_lr = std::max(H.max_lr, std::max(t.size[a], t.size[c]));
    H.lr_pairs += (int64_t)t.size[a] * t.size[c];
    cnt[a + 1]++;
  }
  // low-rank blocks grouped by target cluster (partition order within a group)
  for (int64_t c = 0; c < nc; ++c) cnt[c + 1] += cnt[c];
  std::vector<int32_t> tblk(H.n_lr);
  {
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (int64_t b = 0; b < H.n_lr; ++b) tblk[pos[LR[2 * b]]++] = (int32_t)b;
  }
  // a CTA of the apply takes at most kGroupBlocks of a target's blocks: the groups of a large
  // target would otherwise serialise many blocks in one CTA while few CTAs fill the GPU (one per
  // target cluster: 490 CTAs on 5920 triangles, 26 % of the warps active)
  std::vector<int4> tgrp;
  for (int64_t c = 0; c < nc; ++c)
    for (int64_t q = cnt[c]; q < cnt[c + 1]; q += kGroupBlocks)
      tgrp.push_back(make_int4(t.begin[c], t.size[c], (int)q, (int)std::min<int64_t>(kGroupBlocks, cnt[c + 1] - q)));
  H.n_tg = (int64_t)tgrp.size();
  // dense blocks grouped by target leaf
  std::vector<int64_t> dc(nc + 1, 0);
  H.dn_pairs = 0;
  H.max_leaf = 1;
  for (int64_t b = 0; b < H.n_dn; ++b) {
    const int32_t a = DN[2 * b], c = DN[2 * b + 1];
    dc[a + 1]++;
    H.dn_pairs += (int64_t)t.size[a] * t.size[c];
    H.max_leaf = std::max(H.max_leaf, std::max(t.size[a], t.size[c]));
  }
  for (int64_t c = 0; c < nc; ++c) dc[c + 1] += dc[c];
  std::vector<int2> dsrc(H.n_dn);
  {
    std::vector<int64_t> pos(dc.begin(), dc.end() - 1);
    for (int64_t b = 0; b < H.n_dn; ++b) {
      const int32_t c = DN[2 * b + 1];
      dsrc[pos[DN[2 * b]]++] = make_int2(t.begin[c], t.size[c]);
    }
  }
  std::vector<int4> dgrp;
  for (int64_t c = 0; c < nc; ++c)
    for (int64_t q = dc[c]; q < dc[c + 1]; q += kGroupBlocks)
      dgrp.push_back(make_int4(t.begin[c], t.size[c], (int)q, (int)std::min<int64_t>(kGroupBlocks, dc[c + 1] - q)));
  H.n_dg = (int64_t)dgrp.size();
  upload(ctx, H.perm, t.perm);
  upload(ctx, H.lr, lr);
  upload(ctx, H.tblk, tblk);
  upload(ctx, H.tgrp, tgrp);
  upload(ctx, H.dsrc, dsrc);
  upload(ctx, H.dgrp, dgrp);
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
  H.info.clusters = nc;
  H.info.lowrank_blocks = H.n_lr;
  H.info.dense_blocks = H.n_dn;
  H.info.lowrank_pairs = H.lr_pairs;
  H.info.dense_pairs = H.dn_pairs;
  H.have_structure = true;
}

static void release_factors(HMat& H) {
  H.chunks.clear();
  H.built = false;
  H.F = 0;
}

// Cross approximations of every (low-rank block, frequency) of the current frequency set, in
// batches whose scratch fits a fixed budget; each batch's ranks come back to the host, which
// sizes one storage chunk for the batch and launches the copy into it.
static void build_factors(bem_ctx* ctx) {
  HMat& H = ctx->hm;
  ensure_structure(ctx);
  release_factors(H);
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t F = ctx->fs.F, nlr = H.n_lr;
  const int kmax = H.prm.max_rank;
  const int nmax = 3 * H.max_lr;
  std::vector<int32_t> rank_h((size_t)std::max<int64_t>(F * nlr, 1), 0);
  std::vector<float2*> fptr_h((size_t)std::max<int64_t>(F * nlr, 1), nullptr);
  H.info.rank_sum = 0;
  H.info.rank_max = 0;
  H.info.factor_bytes = 0;
  H.capped.reserve(sizeof(int32_t));
  BEM_CUDA(cudaMemsetAsync(H.capped.p, 0, sizeof(int32_t), ctx->stream));
  const std::vector<int32_t>& LR = H.part.lowrank;
  const hm::Tree& t = H.tree;
  constexpr int64_t kBudget = (int64_t)1 << 28;  // float2 entries of scratch per batch (2 GiB)
  constexpr int64_t kMaxItems = (int64_t)1 << 20;
  const size_t smem = sizeof(cx<float>) * 2 * nmax + nmax;
  BEM_CUDA(cudaFuncSetAttribute(aca_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  AcaArgs a;
  a.g = make_geo(ctx);
  a.lr = H.lr.as<int4>();
  a.fc = ctx->fs.fc32.as<FreqC<float>>();
  a.kmax = kmax;
  a.nmax = nmax;
  a.eps2 = (float)(H.prm.eps * H.prm.eps);
  a.capped = H.capped.as<int32_t>();
  ProfScope ps(ctx, PK_HBUILD, F);
  std::vector<AcaItem> items;
  std::vector<int32_t> brank;
  std::vector<float2*> dst;
  int64_t next = 0;
  const int64_t total = F * nlr;
  {
    // buffers sized once, so that no batch frees memory a previous batch's copy still reads
    int64_t need_all = 0;
    for (int64_t b = 0; b < nlr; ++b) need_all += (int64_t)kmax * 3 * (t.size[LR[2 * b]] + t.size[LR[2 * b + 1]]);
    need_all *= F;
    const int64_t max_item = (int64_t)kmax * 6 * H.max_lr;
    const int64_t nitems = std::min<int64_t>(total, kMaxItems);
    H.scratch.reserve(sizeof(float2) * std::max<int64_t>(std::min(need_all, std::max(kBudget, max_item)), 1));
    H.items.reserve(sizeof(AcaItem) * std::max<int64_t>(nitems, 1));
    H.brank.reserve(sizeof(int32_t) * std::max<int64_t>(nitems, 1));
    H.dst.reserve(sizeof(float2*) * std::max<int64_t>(nitems, 1));
  }
  const int64_t scratch_cap = (int64_t)(H.scratch.bytes / sizeof(float2));
  while (next < total) {
    BEM_CUDA(cudaStreamSynchronize(ctx->stream));  // the previous batch's copy has finished
    items.clear();
    int64_t used = 0;
    while (next < total && (int64_t)items.size() < kMaxItems) {
      const int32_t f = (int32_t)(next / nlr), b = (int32_t)(next % nlr);
      const int64_t need = (int64_t)kmax * 3 * (t.size[LR[2 * b]] + t.size[LR[2 * b + 1]]);
      if (!items.empty() && used + need > scratch_cap) break;
      items.push_back(AcaItem{b, f, used});
      used += need;
      ++next;
    }
    const int64_t nb = (int64_t)items.size();
    BEM_CUDA(cudaMemcpyAsync(H.items.p, items.data(), sizeof(AcaItem) * nb, cudaMemcpyHostToDevice, ctx->stream));
    a.items = H.items.as<AcaItem>();
    a.scratch = H.scratch.as<float2>();
    a.rank = H.brank.as<int32_t>();
    aca_kernel<<<(unsigned)nb, kAcaThreads, smem, ctx->stream>>>(a);
    BEM_LAUNCHED();
    ctx->launches++;
    brank.resize(nb);
    BEM_CUDA(cudaMemcpyAsync(brank.data(), a.rank, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, ctx->stream));
    BEM_CUDA(cudaStreamSynchronize(ctx->stream));
    int64_t bytes = 0;
    for (int64_t q = 0; q < nb; ++q) {
      const int32_t b = items[q].blk;
      bytes += (int64_t)sizeof(float2) * brank[q] * 3 * (t.size[LR[2 * b]] + t.size[LR[2 * b + 1]]);
    }
    dst.assign(nb, nullptr);
    if (bytes > 0) {
      H.chunks.emplace_back(new DevBuf());
      DevBuf& ch = *H.chunks.back();
      ch.reserve(bytes);
      float2* p = ch.as<float2>();
      for (int64_t q = 0; q < nb; ++q) {
        const int32_t b = items[q].blk;
        dst[q] = p;
        p += (int64_t)brank[q] * 3 * (t.size[LR[2 * b]] + t.size[LR[2 * b + 1]]);
      }
      BEM_CUDA(cudaMemcpyAsync(H.dst.p, dst.data(), sizeof(float2*) * nb, cudaMemcpyHostToDevice, ctx->stream));
      CopyArgs c;
      c.lr = a.lr;
      c.items = a.items;
      c.scratch = a.scratch;
      c.rank = a.rank;
      c.dst = H.dst.as<float2*>();
      c.perm = a.g.perm;
      c.bc = a.g.bc;
      c.inv_cscale = 1.f / a.g.cscale;
      c.kmax = kmax;
      copy_factors_kernel<<<(unsigned)nb, 256, 0, ctx->stream>>>(c);
      BEM_LAUNCHED();
      ctx->launches++;
      H.info.factor_bytes += bytes;
    }
    for (int64_t q = 0; q < nb; ++q) {
      const int64_t slot = (int64_t)items[q].f * nlr + items[q].blk;
      rank_h[slot] = brank[q];
      fptr_h[slot] = brank[q] > 0 ? dst[q] : nullptr;
      H.info.rank_sum += brank[q];
      H.info.rank_max = std::max(H.info.rank_max, brank[q]);
    }
  }
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
  upload(ctx, H.rank, rank_h);
  upload(ctx, H.fptr, fptr_h);
  int32_t capped = 0;
  BEM_CUDA(cudaMemcpyAsync(&capped, H.capped.p, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  BEM_CUDA(cudaStreamSynchronize(ctx->stream));
  H.info.capped = capped;
  H.info.frequencies = F;
  H.info.seconds_build = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  H.info.builds++;
  H.F = F;
  H.built = true;
}

bool hm_active(bem_ctx* ctx) { return ctx->hm.prm.enable != 0 && ctx->mesh.ne > 0; }

void hm_invalidate(bem_ctx* ctx, bool structure) {
  HMat& H = ctx->hm;
  release_factors(H);
  if (structure) H.have_structure = false;
}

void hm_far32(bem_ctx* ctx, const cx<float>* x, int64_t nfl) {
  HMat& H = ctx->hm;
  if (!H.built || H.F != ctx->fs.F) build_factors(ctx);
  BEM_REQUIRE(nfl <= 65535, "at most 65535 frequencies per H-matrix application");
  ProfScope ps(ctx, PK_HAPPLY, nfl);
  if (H.n_dg > 0) {
    DenseArgs d;
    d.g = make_geo(ctx);
    d.dgrp = H.dgrp.as<int4>();
    d.dsrc = H.dsrc.as<int2>();
    d.fc = ctx->fs.fc32.as<FreqC<float>>();
    d.x = x;
    d.yacc = ctx->yacc.as<double>();
    d.flist = ctx->flist_d.as<int32_t>();
    d.ne = ctx->mesh.ne;
    dense_apply_kernel<<<dim3((unsigned)H.n_dg, (unsigned)nfl), kDenseThreads, 0, ctx->stream>>>(d);
    BEM_LAUNCHED();
    ctx->launches++;
  }
  if (H.n_tg > 0) {
    LowRankArgs l;
    l.perm = H.perm.as<int32_t>();
    l.lr = H.lr.as<int4>();
    l.tgrp = H.tgrp.as<int4>();
    l.tblk = H.tblk.as<int32_t>();
    l.rank = H.rank.as<int32_t>();
    l.fptr = H.fptr.as<const float2*>();
    l.x = x;
    l.yacc = ctx->yacc.as<double>();
    l.flist = ctx->flist_d.as<int32_t>();
    l.ne = ctx->mesh.ne;
    l.n_lr = H.n_lr;
    l.nmax = 3 * H.max_lr;
    const size_t smem = sizeof(cx<float>) * 2 * l.nmax;
    BEM_CUDA(cudaFuncSetAttribute(lowrank_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    lowrank_apply_kernel<<<dim3((unsigned)H.n_tg, (unsigned)nfl), kApplyThreads, smem, ctx->stream>>>(l);
    BEM_LAUNCHED();
    ctx->launches++;
  }
}

}  // namespace bem

extern "C" {

int bem_default_hmatrix_params(bem_hmatrix_params* p) {
  if (!p) return BEM_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof *p);
  p->enable = 0;
  p->leaf = 32;
  p->max_block = 512;
  p->max_rank = 96;
  p->eta = 2.0;
  p->eps = 1e-4;
  p->max_freqs = 0;
  return BEM_OK;
}

int bem_set_hmatrix(bem_ctx* ctx, const bem_hmatrix_params* p) {
  return bem::guarded_call(ctx, [&] {
    bem_hmatrix_params q;
    bem_default_hmatrix_params(&q);
    if (p) {
      bem::check_params(*p);
      q = *p;
    }
    ctx->hm.prm = q;
    bem::hm_invalidate(ctx, true);
    ctx->hm.info = bem_hmatrix_info{};
  });
}

int bem_get_hmatrix_info(bem_ctx* ctx, bem_hmatrix_info* out) {
  return bem::guarded_call(ctx, [&] {
    BEM_REQUIRE(out, "null output");
    if (bem::hm_active(ctx)) bem::ensure_structure(ctx);
    *out = ctx->hm.info;
  });
}

int bem_hmatrix_partition(const double* verts, int64_t nv, const int32_t* tris, int64_t ne,
                          const bem_hmatrix_params* p, int32_t* perm, int32_t* clusters,
                          int64_t cap_clusters, int32_t* lowrank, int64_t cap_lowrank,
                          int32_t* dense, int64_t cap_dense, int64_t* counts) {
  try {
    BEM_REQUIRE(verts && tris && p && counts, "null argument");
    BEM_REQUIRE(nv > 0 && ne > 0 && ne < ((int64_t)1 << 31), "mesh sizes out of range");
    bem::check_params(*p);
    for (int64_t k = 0; k < 3 * nv; ++k) BEM_REQUIRE(std::isfinite(verts[k]), "non-finite vertex");
    bem::hm::Tree t;
    bem::hm::Partition part;
    bem::hm::cluster_tree(verts, nv, tris, ne, p->leaf, t);
    bem::hm::block_partition(t, p->eta, p->max_block, part);
    const int64_t nc = t.n(), nl = (int64_t)part.lowrank.size() / 2, nd = (int64_t)part.dense.size() / 2;
    if (perm) std::memcpy(perm, t.perm.data(), sizeof(int32_t) * ne);
    if (clusters && cap_clusters >= nc)
      for (int64_t c = 0; c < nc; ++c) {
        clusters[2 * c] = t.begin[c];
        clusters[2 * c + 1] = t.size[c];
      }
    if (lowrank && cap_lowrank >= nl && nl) std::memcpy(lowrank, part.lowrank.data(), sizeof(int32_t) * 2 * nl);
    if (dense && cap_dense >= nd && nd) std::memcpy(dense, part.dense.data(), sizeof(int32_t) * 2 * nd);
    counts[0] = nc;
    counts[1] = nl;
    counts[2] = nd;
    return BEM_OK;
  } catch (const bem::Error& e) {
    bem::set_global_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    bem::set_global_error(e.what());
    return BEM_ERR_INVALID_ARG;
  }
}

}  // extern "C"
