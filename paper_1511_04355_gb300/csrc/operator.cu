// Matrix-free application of the discretised boundary integral operator, batched over
// frequencies (Sec. 2.1, Eqs. (bie), (Aa_b)):
//     y_i(s) = sum_e  Op_ie(s) x_e(s),   i, e = 1 .. n_e,  for every s in the batch,
// where Op_ie is, per source column e,
//     A (system):  traction given -> 1/2 delta_ie I + H_ie(s),  displacement given -> -G_ie(s)
//     K (data)  :  traction given -> G_ie(s),  displacement given -> -(1/2 delta_ie I + H_ie(s))
// so that A(s) a(s) = b(s) = K(s) (known boundary data).  Three kernels:
//   far_kernel   : 4-point rule over ALL sources e != i, kernels evaluated on the fly.  One
//                  thread per collocation point, FT frequencies per thread (the geometry of a
//                  source point is shared by the FT frequencies), source elements staged in
//                  shared memory tile by tile, FP32 (or FP64) partial sums per tile flushed to
//                  FP64 accumulators in shared memory.
//   near_kernel  : for sources in the near list, the 7-point rule minus the 4-point rule (the
//                  far kernel already added the latter), plus the own-element 3x3 block.
//   precond      : right block-Jacobi, y_i = A_ii^{-1} x_i.
#include <algorithm>

#include "kernel_math.cuh"

namespace bem {

template <class R>
struct V4;
template <>
struct V4<float> {
  using T = float4;
};
template <>
struct V4<double> {
  using T = D4;
};

// ------------------------------------------------------------------------------- far field
template <class R>
struct FarArgs {
  const typename V4<R>::T* q4;  // [ne][4] (x, y, z, w * area)
  const typename V4<R>::T* cen; // [ne] centroid (x, y, z, -)
  const typename V4<R>::T* nrm; // [ne] normal (x, y, z, -)
  const float4* q4lo;           // FP32 only: low parts of q4 and of the centroids
  const float4* cenlo;
  const int8_t* bc;             // [ne] or null (all traction-given)
  int which;                    // BEM_APPLY_A / BEM_APPLY_K (apply mode)
  const cx<R>* x;               // [F][ne][3]
  const double* bcv;            // [ne][3] known-data pattern (residual mode)
  const cx<double>* pfac;       // [F] time-profile factor (residual mode)
  double* yacc;                 // [F][ne][3] complex FP64 accumulator (atomic adds)
  const FreqC<R>* fc;           // [F]
  const int32_t* flist;         // frequencies to compute (the active ones), nfl entries
  const FarGroup* groups;       // recurrence kernel: one per blockIdx.y, its run of list entries
  int64_t nfl;
  int64_t chunk;                // sources per split (multiple of the tile size)
  int64_t ne, F;
  MatC<R> m;
};

// code of a source column: |code| = 1 -> T kernel, 2 -> U kernel; sign = column sign
__device__ __forceinline__ float column_code(const int8_t* bc, int64_t e, int which) {
  const int b = bc ? (int)bc[e] : 0;
  const int useU = b ^ which;
  const float sign = b ? -1.f : 1.f;
  return sign * (useU ? 2.f : 1.f);
}

// T-kernel contribution of one source point to the three output components:
//   o_c += cw [A (dr/dn v_c + (rh.v) n_c) + rh_c (q1 (n.v) + q2 dr/dn (rh.v))]
template <class R>
__device__ __forceinline__ void t_contract(const TCoef<R>& T, R cw, R drdn, R rh0, R rh1, R rh2,
                                           R n0, R n1, R n2, cx<R> v0, cx<R> v1, cx<R> v2,
                                           cx<R> nv, cx<R>* o) {
  const cx<R> rv = mk(rh0 * v0.r + rh1 * v1.r + rh2 * v2.r, rh0 * v0.i + rh1 * v1.i + rh2 * v2.i);
  const cx<R> t1 = (cw * drdn) * T.A;
  const cx<R> t2 = (cw * T.A) * rv;
  const cx<R> t3 = cw * cfma(T.q1, nv, drdn * (T.q2 * rv));
  o[0] = cfma(t1, v0, axpy(n0, t2, axpy(rh0, t3, o[0])));
  o[1] = cfma(t1, v1, axpy(n1, t2, axpy(rh1, t3, o[1])));
  o[2] = cfma(t1, v2, axpy(n2, t2, axpy(rh2, t3, o[2])));
}

// U-kernel contribution: o_c += cu [(E_s - J) v_c - (P - 3J) rh_c (rh.v)]
template <class R>
__device__ __forceinline__ void u_contract(const Radial<R>& K, R cu, R rh0, R rh1, R rh2, cx<R> v0,
                                           cx<R> v1, cx<R> v2, cx<R>* o) {
  const cx<R> psi = cu * (K.Es - K.J);
  const cx<R> rv = mk(rh0 * v0.r + rh1 * v1.r + rh2 * v2.r, rh0 * v0.i + rh1 * v1.i + rh2 * v2.i);
  const cx<R> crv = (cu * axpy(R(-3), K.J, K.P)) * rv;
  o[0] = cfma(psi, v0, axpy(-rh0, crv, o[0]));
  o[1] = cfma(psi, v1, axpy(-rh1, crv, o[1]));
  o[2] = cfma(psi, v2, axpy(-rh2, crv, o[2]));
}

// Far-field kernel (FP64: the plain-FP64 path and the native FP64 residual).  Apply mode
// (RESID = false): y = Op x with Op = A or K, one kernel (T or U) per source column.  Residual mode (RESID = true): y = K k - A x with k = profile(s) * known
// data; every source contributes through both kernels, T applied to vT and U to vU where
// (vT, vU) = (-x_e, k_e) for traction-given and (-k_e, x_e) for displacement-given columns.
// e^{-i theta} with theta = (w_hi + w_lo)(r + r_lo), |theta| <= 1.5 (the host admits a group
// only then): theta in float-float, cos and sin of its high part by their Taylor series (terms
// to theta^12 / theta^13, truncation < 4e-9), the low part added to first order.  Accurate to
// about an ulp: the recurrence multiplies this factor up to FT - 1 times.
__device__ __forceinline__ cx<float> step_factor(float w_hi, float w_lo, float r, float r_lo) {
  const float th = w_hi * r;
  const float tl = fmaf(w_hi, r, -th) + fmaf(w_hi, r_lo, w_lo * r);
  const float t = th * th;
  float c = fmaf(t, 1.f / 479001600.f, -1.f / 3628800.f);
  c = fmaf(t, c, 1.f / 40320.f);
  c = fmaf(t, c, -1.f / 720.f);
  c = fmaf(t, c, 1.f / 24.f);
  c = fmaf(t, c, -0.5f);
  c = fmaf(t, c, 1.f);
  float sn = fmaf(t, -1.f / 6227020800.f, 1.f / 39916800.f);
  sn = fmaf(t, sn, -1.f / 362880.f);
  sn = fmaf(t, sn, 1.f / 5040.f);
  sn = fmaf(t, sn, -1.f / 120.f);
  sn = fmaf(t, sn, 1.f / 6.f);
  sn = fmaf(-t * th, sn, th);
  // cos(th + tl) ~ c - sn tl, sin(th + tl) ~ sn + c tl
  return mk(fmaf(-sn, tl, c), -fmaf(c, tl, sn));
}

template <class R, int TB, int S, int FT, bool RESID>
__global__ void __launch_bounds__(TB) far_kernel(const FarArgs<R> a) {
  using V = typename V4<R>::T;
  constexpr int NV = RESID ? 7 : 4;                                    // cx per (source, freq)
  extern __shared__ __align__(32) unsigned char smem_raw[];
  // accumulators: per-tile partial sums (registers) are added into R-precision sums here, then
  // into the FP64 result with one atomic add per output at the end
  R* acc = reinterpret_cast<R*>(smem_raw);                            // [6 FT][TB]
  V* sq = reinterpret_cast<V*>(smem_raw + sizeof(R) * 6 * FT * TB);   // [S][4]
  V* sn = sq + 4 * S;                                                  // [S]
  cx<R>* sv = reinterpret_cast<cx<R>*>(sn + S);                       // [S][FT][NV]
  FreqC<R>* sfc = reinterpret_cast<FreqC<R>*>(sv + NV * FT * S);      // [FT]

  const int tid = threadIdx.x;
  const int64_t g0 = (int64_t)blockIdx.y * FT;   // position in the frequency list
  const int nf = (int)min((int64_t)FT, a.nfl - g0);
  const unsigned mask = (1u << nf) - 1u;
  const int64_t src0 = (int64_t)blockIdx.z * a.chunk;
  const int64_t src1 = min(a.ne, src0 + a.chunk);
  const int64_t i = (int64_t)blockIdx.x * TB + tid;
  const bool valid = i < a.ne;
  R xi0 = 0, xi1 = 0, xi2 = 0;
  if (valid) {
    const V c = a.cen[i];
    xi0 = c.x;
    xi1 = c.y;
    xi2 = c.z;
  }
  if (tid < FT) {
    if (tid < nf) sfc[tid] = a.fc[a.flist[g0 + tid]];
    else sfc[tid] = FreqC<R>{};
  }
#pragma unroll
  for (int k = 0; k < 6 * FT; ++k) acc[k * TB + tid] = R(0);
  const MatC<R>& m = a.m;
  __syncthreads();
  const R inv4pi = R(kInv4Pi);

  for (int64_t e0 = src0; e0 < src1; e0 += S) {
    const int ns = (int)min((int64_t)S, src1 - e0);
    __syncthreads();
    for (int t = tid; t < 4 * ns; t += TB) sq[t] = a.q4[4 * e0 + t];
    for (int t = tid; t < ns; t += TB) {
      V n = a.nrm[e0 + t];
      n.w = (R)column_code(a.bc, e0 + t, a.which);
      sn[t] = n;
    }
    for (int t = tid; t < ns * FT; t += TB) {
      const int e = t / FT, k = t % FT;
      const int64_t ge = e0 + e;
      cx<R> v0 = mk(R(0), R(0)), v1 = v0, v2 = v0, k0 = v0, k1 = v0, k2 = v0;
      if (k < nf) {
        const int64_t f = a.flist[g0 + k];
        const cx<R>* xv = a.x + (f * a.ne + ge) * 3;
        v0 = xv[0];
        v1 = xv[1];
        v2 = xv[2];
        if (RESID) {
          const cx<double> pf = a.pfac[f];
          const double* kv = a.bcv + 3 * ge;
          k0 = mk((R)(pf.r * kv[0]), (R)(pf.i * kv[0]));
          k1 = mk((R)(pf.r * kv[1]), (R)(pf.i * kv[1]));
          k2 = mk((R)(pf.r * kv[2]), (R)(pf.i * kv[2]));
        }
      }
      const V n = a.nrm[ge];
      cx<R>* o = sv + NV * (e * FT + k);
      if (RESID) {
        const bool dir = a.bc && a.bc[ge] == BEM_BC_DISPLACEMENT;
        const cx<R> t0 = dir ? k0 : v0, t1 = dir ? k1 : v1, t2 = dir ? k2 : v2;
        const cx<R> u0 = dir ? v0 : k0, u1 = dir ? v1 : k1, u2 = dir ? v2 : k2;
        o[0] = R(-1) * t0;
        o[1] = R(-1) * t1;
        o[2] = R(-1) * t2;
        o[3] = mk(-(n.x * t0.r + n.y * t1.r + n.z * t2.r), -(n.x * t0.i + n.y * t1.i + n.z * t2.i));
        o[4] = u0;
        o[5] = u1;
        o[6] = u2;
      } else {
        o[0] = v0;
        o[1] = v1;
        o[2] = v2;
        o[3] = mk(n.x * v0.r + n.y * v1.r + n.z * v2.r, n.x * v0.i + n.y * v1.i + n.z * v2.i);
      }
    }
    __syncthreads();

    cx<R> part[FT][3];
#pragma unroll
    for (int k = 0; k < FT; ++k) part[k][0] = part[k][1] = part[k][2] = mk(R(0), R(0));

    for (int e = 0; e < ns; ++e) {
      const V nn = sn[e];
      const bool self = (e0 + e == i);
      const bool isU = fabs((double)nn.w) > 1.5;
      const R sign = RESID ? R(1) : (nn.w > 0 ? R(1) : R(-1));
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        const V p = sq[4 * e + q];
        const Dist<R> D = distance(p.x, p.y, p.z, make_float4(0.f, 0.f, 0.f, 0.f), xi0, xi1, xi2,
                                   make_float4(0.f, 0.f, 0.f, 0.f), self);
        const R r = D.r, rinv = D.rinv;
        const R inv_r2 = rinv * rinv;
        const R rh0 = D.dx * rinv, rh1 = D.dy * rinv, rh2 = D.dz * rinv;
        const R w = self ? R(0) : p.w * sign;
        const R drdn = rh0 * nn.x + rh1 * nn.y + rh2 * nn.z;
        const R cw = w * inv_r2 * inv4pi;
        const R cu = w * rinv * m.inv4pimu;
        if (RESID || !isU) {
#pragma unroll
          for (int k = 0; k < FT; ++k) {
            if (!((mask >> k) & 1u)) continue;
            const cx<R>* v = sv + NV * (e * FT + k);
            const Radial<R> K = radial(r, inv_r2, sfc[k], m);
            const TCoef<R> T = tcoef(K, m);
            t_contract(T, cw, drdn, rh0, rh1, rh2, nn.x, nn.y, nn.z, v[0], v[1], v[2], v[3], part[k]);
            if (RESID) u_contract(K, cu, rh0, rh1, rh2, v[4], v[5], v[6], part[k]);
          }
        } else {
#pragma unroll
          for (int k = 0; k < FT; ++k) {
            if (!((mask >> k) & 1u)) continue;
            const cx<R>* v = sv + NV * (e * FT + k);
            const Radial<R> K = radial(r, inv_r2, sfc[k], m);
            u_contract(K, cu, rh0, rh1, rh2, v[0], v[1], v[2], part[k]);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < FT; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[(6 * k + 2 * c) * TB + tid] += part[k][c].r;
        acc[(6 * k + 2 * c + 1) * TB + tid] += part[k][c].i;
      }
  }
  if (!valid) return;
#pragma unroll
  for (int k = 0; k < FT; ++k) {
    if (!((mask >> k) & 1u)) continue;
    double* yo = a.yacc + ((int64_t)a.flist[g0 + k] * a.ne + i) * 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) atomicAdd(yo + c, (double)acc[(6 * k + c) * TB + tid]);
  }
}

// FP32 far field in apply mode (y = A x or K x), frequency-outer loop: for each source element
// the geometry of its 4 quadrature points is formed once and kept in registers, then for each of
// the CTA's frequencies the 4 points are summed.  The terms that multiply the element's source
// values v and normal n, sum_q t1_q v + sum_q t2_q n (T columns) or sum_q psi_q v (U columns),
// are accumulated over the points and applied once per element; only the rh_q term stays per
// point.  REC: equally spaced group, E(s_k) = E(s_{k-1}) e^{-i delta r / c} per point.
// Shared memory: the accumulators, the source tile (points, low parts, normals, values) and the
// frequency constants (far_smem<float, ..., RESID = false>).
template <int TB, int S, int FT, bool REC>
__global__ void __launch_bounds__(TB) far32_kernel(const FarArgs<float> a) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  float* acc = reinterpret_cast<float*>(smem_raw);                            // [6 FT][TB]
  float4* sq = reinterpret_cast<float4*>(smem_raw + sizeof(float) * 6 * FT * TB);  // [S][4]
  float4* sn = sq + 4 * S;                                                     // [S]
  float4* sql = sn + S;                                                        // [S][4]
  cx<float>* sv = reinterpret_cast<cx<float>*>(sql + 4 * S);                  // [S][FT][4]
  FreqC<float>* sfc = reinterpret_cast<FreqC<float>*>(sv + 4 * FT * S);       // [FT]

  const int tid = threadIdx.x;
  FarGroup grp{};
  if constexpr (REC) grp = a.groups[blockIdx.y];
  const int64_t g0 = REC ? (int64_t)grp.start : (int64_t)blockIdx.y * FT;
  const int nf = REC ? grp.count : (int)min((int64_t)FT, a.nfl - g0);
  const int64_t src0 = (int64_t)blockIdx.z * a.chunk;
  const int64_t src1 = min(a.ne, src0 + a.chunk);
  const int64_t i = (int64_t)blockIdx.x * TB + tid;
  const bool valid = i < a.ne;
  float xi0 = 0, xi1 = 0, xi2 = 0;
  float4 xil = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) {
    const float4 c = a.cen[i];
    xi0 = c.x;
    xi1 = c.y;
    xi2 = c.z;
    xil = a.cenlo[i];
  }
  if (tid < FT) {
    if (tid < nf) sfc[tid] = a.fc[a.flist[g0 + tid]];
    else sfc[tid] = FreqC<float>{};
  }
#pragma unroll
  for (int k = 0; k < 6 * FT; ++k) acc[k * TB + tid] = 0.f;
  const MatC<float>& m = a.m;
  __syncthreads();
  bool same_re = true;
  for (int k = 1; k < nf; ++k) same_re = same_re && sfc[k].a.r == sfc[0].a.r;
  const float re_s = -sfc[0].a.r;
  const float re_p = -(sfc[0].a.r * m.beta);
  const float inv4pi = (float)kInv4Pi;

  for (int64_t e0 = src0; e0 < src1; e0 += S) {
    const int ns = (int)min((int64_t)S, src1 - e0);
    __syncthreads();
    for (int t = tid; t < 4 * ns; t += TB) sq[t] = a.q4[4 * e0 + t];
    for (int t = tid; t < 4 * ns; t += TB) sql[t] = a.q4lo[4 * e0 + t];
    for (int t = tid; t < ns; t += TB) {
      float4 n = a.nrm[e0 + t];
      n.w = column_code(a.bc, e0 + t, a.which);
      sn[t] = n;
    }
    for (int t = tid; t < ns * FT; t += TB) {
      const int e = t / FT, k = t % FT;
      const int64_t ge = e0 + e;
      cx<float> v0 = mk(0.f, 0.f), v1 = v0, v2 = v0;
      if (k < nf) {
        const cx<float>* xv = a.x + ((int64_t)a.flist[g0 + k] * a.ne + ge) * 3;
        v0 = xv[0];
        v1 = xv[1];
        v2 = xv[2];
      }
      const float4 n = a.nrm[ge];
      cx<float>* o = sv + 4 * (e * FT + k);
      o[0] = v0;
      o[1] = v1;
      o[2] = v2;
      o[3] = mk(n.x * v0.r + n.y * v1.r + n.z * v2.r, n.x * v0.i + n.y * v1.i + n.z * v2.i);
    }
    __syncthreads();

    for (int e = 0; e < ns; ++e) {
      const float4 nn = sn[e];
      const bool self = (e0 + e == i);
      const bool isU = fabsf(nn.w) > 1.5f;
      const float sign = nn.w > 0 ? 1.f : -1.f;
      // the element's 4 points: distance, direction, weights, amplitudes (and recurrence state)
      float r[4], rlo[4], ir2[4], rh0[4], rh1[4], rh2[4], drdn[4], cwu[4], ams[4], amp[4];
      cx<float> Es[4], Ep[4], ws[4], wp[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 p = sq[4 * e + q];
        const Dist<float> D = distance(p.x, p.y, p.z, sql[4 * e + q], xi0, xi1, xi2, xil, self);
        r[q] = D.r;
        rlo[q] = D.r_lo;
        ir2[q] = D.rinv * D.rinv;
        rh0[q] = D.dx * D.rinv;
        rh1[q] = D.dy * D.rinv;
        rh2[q] = D.dz * D.rinv;
        drdn[q] = rh0[q] * nn.x + rh1[q] * nn.y + rh2[q] * nn.z;
        const float w = self ? 0.f : p.w * sign;
        cwu[q] = isU ? w * D.rinv * m.inv4pimu : w * ir2[q] * inv4pi;
        ams[q] = amp[q] = -1.f;
        if (same_re) {
          ams[q] = __expf(re_s * r[q]);
          amp[q] = __expf(re_p * r[q]);
        }
        if constexpr (REC) {
          radial_exps(r[q], sfc[0], m, rlo[q], ams[q], amp[q], Es[q], Ep[q]);
          ws[q] = step_factor(grp.ws_hi, grp.ws_lo, r[q], rlo[q]);
          wp[q] = step_factor(grp.wp_hi, grp.wp_lo, r[q], rlo[q]);
        }
      }
#pragma unroll 1
      for (int k = 0; k < nf; ++k) {
        const FreqC<float>& F = sfc[k];
        const cx<float>* v = sv + 4 * (e * FT + k);
        const cx<float> v0 = v[0], v1 = v[1], v2 = v[2], nv = v[3];
        cx<float> T1 = mk(0.f, 0.f), T2 = T1, o0 = T1, o1 = T1, o2 = T1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          cx<float> es, ep;
          if constexpr (REC) {
            if (k > 0) {
              Es[q] = Es[q] * ws[q];
              Ep[q] = Ep[q] * wp[q];
            }
            es = Es[q];
            ep = Ep[q];
          } else {
            radial_exps(r[q], F, m, rlo[q], ams[q], amp[q], es, ep);
          }
          const Radial<float> K = radial_given(r[q], ir2[q], F, m, es, ep);
          const cx<float> rv = mk(rh0[q] * v0.r + rh1[q] * v1.r + rh2[q] * v2.r,
                                  rh0[q] * v0.i + rh1[q] * v1.i + rh2[q] * v2.i);
          if (!isU) {
            // T: o_c += cw [A (dr/dn v_c + (rh.v) n_c) + rh_c (q1 (n.v) + q2 dr/dn (rh.v))]
            const TCoef<float> T = tcoef(K, m);
            const cx<float> al = cwu[q] * T.A;
            T1 = axpy(drdn[q], al, T1);
            T2 = cfma(al, rv, T2);
            const cx<float> t3 = cwu[q] * cfma(T.q1, nv, drdn[q] * (T.q2 * rv));
            o0 = axpy(rh0[q], t3, o0);
            o1 = axpy(rh1[q], t3, o1);
            o2 = axpy(rh2[q], t3, o2);
          } else {
            // U: o_c += cu [(E_s - J) v_c - (P - 3J) rh_c (rh.v)]
            T1 = T1 + cwu[q] * (K.Es - K.J);
            const cx<float> crv = (cwu[q] * axpy(-3.f, K.J, K.P)) * rv;
            o0 = axpy(-rh0[q], crv, o0);
            o1 = axpy(-rh1[q], crv, o1);
            o2 = axpy(-rh2[q], crv, o2);
          }
        }
        o0 = cfma(T1, v0, axpy(nn.x, T2, o0));
        o1 = cfma(T1, v1, axpy(nn.y, T2, o1));
        o2 = cfma(T1, v2, axpy(nn.z, T2, o2));
        float* ac = acc + (6 * k) * TB + tid;
        ac[0] += o0.r;
        ac[TB] += o0.i;
        ac[2 * TB] += o1.r;
        ac[3 * TB] += o1.i;
        ac[4 * TB] += o2.r;
        ac[5 * TB] += o2.i;
      }
    }
  }
  if (!valid) return;
  for (int k = 0; k < nf; ++k) {
    double* yo = a.yacc + ((int64_t)a.flist[g0 + k] * a.ne + i) * 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) atomicAdd(yo + c, (double)acc[(6 * k + c) * TB + tid]);
  }
}

template <class R, int TB, int S, int FT, bool RESID>
static size_t far_smem() {
  using V = typename V4<R>::T;
  return sizeof(R) * 6 * FT * TB + sizeof(V) * 5 * S + (sizeof(R) == 4 ? sizeof(float4) * 4 * S : 0) +
         sizeof(cx<R>) * (RESID ? 7 : 4) * FT * S + sizeof(FreqC<R>) * FT;
}

// ------------------------------------------------------------------------------- near field
template <class R>
struct NearArgs {
  const typename V4<R>::T* q4;
  const typename V4<R>::T* q7;
  const typename V4<R>::T* cen;
  const typename V4<R>::T* nrm;
  const int32_t *ptr, *col;
  const int8_t* bc;
  int which;
  bool resid;               // residual mode: y = K k - A x
  const double* bcv;        // [ne][3] known-data pattern (residual mode)
  const cx<double>* pfac;   // [F]
  const cx<double>* Tself;  // [F][ne][9]
  const cx<double>* Gself;
  const cx<R>* x;
  cx<R>* y;
  const double* yacc;       // far-field sums [F][ne][3] complex
  const FreqC<R>* fc;
  const int32_t* flist;
  int64_t nfl;
  int64_t ne, F;
  MatC<R> m;
};

// one source point: T contraction with vT (if useT) and U contraction with vU (if useU)
template <class R>
__device__ __forceinline__ void add_point(R xi0, R xi1, R xi2, const typename V4<R>::T& p, R wsign,
                                          const typename V4<R>::T& nn, bool useT, bool useU,
                                          const FreqC<R>& fc, const MatC<R>& m, const cx<R>* vT,
                                          cx<R> nvT, const cx<R>* vU, cx<R>* o) {
  const R dx = p.x - xi0, dy = p.y - xi1, dz = p.z - xi2;
  const R r2 = dx * dx + dy * dy + dz * dz;
  const R rinv = rsqrt_r(r2), r = r2 * rinv, inv_r2 = rinv * rinv;
  const R rh0 = dx * rinv, rh1 = dy * rinv, rh2 = dz * rinv;
  const Radial<R> K = radial(r, inv_r2, fc, m);
  if (useT) {
    const R drdn = rh0 * nn.x + rh1 * nn.y + rh2 * nn.z;
    const R cw = p.w * wsign * inv_r2 * R(kInv4Pi);
    t_contract(tcoef(K, m), cw, drdn, rh0, rh1, rh2, nn.x, nn.y, nn.z, vT[0], vT[1], vT[2], nvT, o);
  }
  if (useU) u_contract(K, p.w * wsign * rinv * m.inv4pimu, rh0, rh1, rh2, vU[0], vU[1], vU[2], o);
}

// WARP = false: one thread per (listed frequency, target), the near sources in sequence (many
// frequencies fill the GPU).  WARP = true: one warp per (listed frequency, target), its lanes
// over the (near source, point) pairs and a shuffle reduction, for launches with few frequencies
// (a single AFS frequency on 6960 triangles launched only 55 blocks of threads and took 0.38 ms).
template <class R, bool WARP>
__global__ void near_kernel(const NearArgs<R> a) {
  using V = typename V4<R>::T;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t t = WARP ? gt >> 5 : gt;
  const int lane = WARP ? (int)(threadIdx.x & 31) : 0;
  if (t >= a.nfl * a.ne) return;  // WARP: the same t for every lane of a warp
  const int64_t f = a.flist[t / a.ne], i = t % a.ne;
  const V c = a.cen[i];
  const FreqC<R> fc = a.fc[f];
  const cx<double> pf = a.resid ? a.pfac[f] : mk(0.0, 0.0);
  cx<R> o[3] = {mk(R(0), R(0)), mk(R(0), R(0)), mk(R(0), R(0))};
  // source vectors of element e: apply mode -> (v, v) with the column's kernel; residual mode
  // -> vT = -x or -k, vU = k or x (see far_kernel)
  auto load = [&](int64_t e, cx<R>* vT, cx<R>& nvT, cx<R>* vU, bool& useT, bool& useU, R& sign) {
    const V nn = a.nrm[e];
    const cx<R>* xv = a.x + (f * a.ne + e) * 3;
    if (!a.resid) {
      const float code = column_code(a.bc, e, a.which);
      useU = fabsf(code) > 1.5f;
      useT = !useU;
      sign = code > 0 ? R(1) : R(-1);
      for (int q = 0; q < 3; ++q) vT[q] = vU[q] = xv[q];
    } else {
      useT = useU = true;
      sign = R(1);
      const bool dir = a.bc && a.bc[e] == BEM_BC_DISPLACEMENT;
      for (int q = 0; q < 3; ++q) {
        const double kv = a.bcv[3 * e + q];
        const cx<R> kq = mk((R)(pf.r * kv), (R)(pf.i * kv));
        vT[q] = R(-1) * (dir ? kq : xv[q]);
        vU[q] = dir ? xv[q] : kq;
      }
    }
    nvT = mk(nn.x * vT[0].r + nn.y * vT[1].r + nn.z * vT[2].r, nn.x * vT[0].i + nn.y * vT[1].i + nn.z * vT[2].i);
  };
  if constexpr (WARP) {
    const int32_t p0 = a.ptr[i];
    const int32_t nwork = (a.ptr[i + 1] - p0) * 11;
    for (int32_t w = lane; w < nwork; w += 32) {
      const int64_t e = a.col[p0 + w / 11];
      const int q = w % 11;
      cx<R> vT[3], vU[3], nvT;
      bool useT, useU;
      R sign;
      load(e, vT, nvT, vU, useT, useU, sign);
      const V nn = a.nrm[e];
      if (q < 7) add_point(c.x, c.y, c.z, a.q7[7 * e + q], sign, nn, useT, useU, fc, a.m, vT, nvT, vU, o);
      else add_point(c.x, c.y, c.z, a.q4[4 * e + (q - 7)], -sign, nn, useT, useU, fc, a.m, vT, nvT, vU, o);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
      for (int off = 16; off > 0; off >>= 1) {
        o[r].r += __shfl_down_sync(0xffffffffu, o[r].r, off);
        o[r].i += __shfl_down_sync(0xffffffffu, o[r].i, off);
      }
    if (lane != 0) return;
  } else {
    for (int32_t p = a.ptr[i]; p < a.ptr[i + 1]; ++p) {
      const int64_t e = a.col[p];
      cx<R> vT[3], vU[3], nvT;
      bool useT, useU;
      R sign;
      load(e, vT, nvT, vU, useT, useU, sign);
      const V nn = a.nrm[e];
      for (int q = 0; q < 7; ++q)
        add_point(c.x, c.y, c.z, a.q7[7 * e + q], sign, nn, useT, useU, fc, a.m, vT, nvT, vU, o);
      for (int q = 0; q < 4; ++q)
        add_point(c.x, c.y, c.z, a.q4[4 * e + q], -sign, nn, useT, useU, fc, a.m, vT, nvT, vU, o);
    }
  }
  // own element from the FP64 singular blocks: H_ii' = 1/2 I + H_ii applied to vT, G_ii to vU
  {
    cx<R> vT[3], vU[3], nvT;
    bool useT, useU;
    R sign;
    load(i, vT, nvT, vU, useT, useU, sign);
    const cx<double>* Hb = a.Tself + (f * a.ne + i) * 9;
    const cx<double>* Gb = a.Gself + (f * a.ne + i) * 9;
    for (int r = 0; r < 3; ++r) {
      cx<R> s = mk(R(0), R(0));
      for (int cc = 0; cc < 3; ++cc) {
        if (useT) {
          cx<double> d = Hb[3 * r + cc];
          if (r == cc) d.r += 0.5;
          s = cfma(sign * mk((R)d.r, (R)d.i), vT[cc], s);
        }
        if (useU) {
          const cx<double> d = Gb[3 * r + cc];
          s = cfma(sign * mk((R)d.r, (R)d.i), vU[cc], s);
        }
      }
      o[r] = o[r] + s;
    }
  }
  cx<R>* yo = a.y + (f * a.ne + i) * 3;
  const double* ya = a.yacc + (f * a.ne + i) * 6;
  for (int r = 0; r < 3; ++r) yo[r] = mk((R)ya[2 * r], (R)ya[2 * r + 1]) + o[r];
}

// ------------------------------------------------------------------------------- precond
template <class R>
__global__ void precond_kernel(const cx<R>* Minv, const cx<R>* x, cx<R>* y, const int32_t* active,
                               int64_t ne, int64_t F) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= F * ne) return;
  const int64_t f = t / ne;
  if (active && !active[f]) return;
  const cx<R>* M = Minv + 9 * t;
  const cx<R>* xv = x + 3 * t;
  const cx<R> v0 = xv[0], v1 = xv[1], v2 = xv[2];
  cx<R>* yo = y + 3 * t;
  for (int r = 0; r < 3; ++r) yo[r] = cfma(M[3 * r + 2], v2, cfma(M[3 * r + 1], v1, M[3 * r] * v0));
}

__global__ void known_data_kernel(const cx<double>* pfac, const double* val, cx<double>* out,
                                  int64_t ne, int64_t F) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= F * ne * 3) return;
  const int64_t f = t / (3 * ne), r = t % (3 * ne);
  out[t] = val[r] * pfac[f];
}

// ------------------------------------------------------------------------------- host side
template <class R>
struct Geo;
template <>
struct Geo<float> {
  static const float4* q4(bem_ctx* c) { return c->mesh.q4_32.as<float4>(); }
  static const float4* q7(bem_ctx* c) { return c->mesh.q7_32.as<float4>(); }
  static const float4* cen(bem_ctx* c) { return c->mesh.c32.as<float4>(); }
  static const float4* nrm(bem_ctx* c) { return c->mesh.n32.as<float4>(); }
  static const FreqC<float>* fc(bem_ctx* c) { return c->fs.fc32.as<FreqC<float>>(); }
  static MatC<float> m(bem_ctx* c) { return mat_constants32(c->mat); }
};
template <>
struct Geo<double> {
  static const D4* q4(bem_ctx* c) { return c->mesh.q4_64.as<D4>(); }
  static const D4* q7(bem_ctx* c) { return c->mesh.q7_64.as<D4>(); }
  static const D4* cen(bem_ctx* c) { return c->mesh.c64.as<D4>(); }
  static const D4* nrm(bem_ctx* c) { return c->mesh.n64.as<D4>(); }
  static const FreqC<double>* fc(bem_ctx* c) { return c->fs.fc64.as<FreqC<double>>(); }
  static MatC<double> m(bem_ctx* c) { return mat_constants64(c->mat); }
};

template <class R>
struct Cfg;
template <>
struct Cfg<float> {  // FP32: 128 targets x 12 frequencies per CTA, 32-element source tiles
  // (12 rather than 8 amortises each element's geometry over more frequencies while 4 CTAs of
  // 54 KB shared memory still fit an SM: 5 % faster on the 5120-triangle cavity; with 16 only
  // 3 CTAs fit, and it was slower than 12)
  static constexpr int TB = 128, S = 32, FT = 12, kPerSM = 4;
};
template <>
struct Cfg<double> {  // FP64: 128 targets x 4 frequencies per CTA, 32-element source tiles
  static constexpr int TB = 128, S = 32, FT = 4, kPerSM = 4;
};

// Device copy of the frequency list (all frequencies when `flist` is null), its grouping into
// CTA frequency groups, and the FP64 far-field accumulator zeroed for the listed frequencies.
// rec_ft > 0 (FP32 operator): the list is reordered into equally spaced runs of at least 4
// frequencies (groups of at most rec_ft, for the recurrence kernel) followed by the remaining
// frequencies (FT per CTA); a run qualifies when its frequencies share Re s, their Im s steps
// agree to 1e-12 relative (FP64) and one step's phase (Im delta / c_s) x the mesh's
// bounding-box diagonal is at most 1.5.  rec_ft = 0: list order, FT per CTA.
int64_t stage_flist(bem_ctx* ctx, const std::vector<int32_t>* flist, int rec_ft) {
  const int64_t F = ctx->fs.F, ne = ctx->mesh.ne;
  std::vector<int32_t>& h = ctx->flist_h;
  if (flist) h = *flist;
  else {
    h.resize(F);
    for (int64_t f = 0; f < F; ++f) h[f] = (int32_t)f;
  }
  const int64_t n = (int64_t)h.size();
  std::vector<FarGroup>& gr = ctx->groups_h;
  gr.clear();
  ctx->rec_entries = 0;
  if (rec_ft > 0 && n > 0) {
    const std::vector<double>& s = ctx->fs.s;
    const MatC<double> m = mat_constants64(ctx->mat);
    std::vector<int32_t> rec, rest;
    std::vector<FarGroup> rg;
    int64_t i = 0;
    while (i < n) {
      int64_t j = i + 1;
      double d = 0.0;
      if (i + 1 < n) {
        const double re0 = s[2 * h[i]], im0 = s[2 * h[i] + 1];
        d = s[2 * h[i + 1] + 1] - im0;
        const bool small = std::fabs(d * m.inv_cs) * ctx->mesh.diam <= 1.5;
        if (d != 0.0 && small && s[2 * h[i + 1]] == re0) {
          j = i + 2;
          while (j < n && j - i < rec_ft && s[2 * h[j]] == re0 &&
                 std::fabs((s[2 * h[j] + 1] - im0) - (double)(j - i) * d) <= 1e-12 * std::fabs(s[2 * h[j] + 1]))
            ++j;
        }
      }
      if (j - i >= 4) {
        FarGroup g{};
        g.start = (int32_t)rec.size();
        g.count = (int32_t)(j - i);
        const double ws = d * m.inv_cs, wp = ws * m.beta;
        g.ws_hi = (float)ws;
        g.ws_lo = (float)(ws - (double)g.ws_hi);
        g.wp_hi = (float)wp;
        g.wp_lo = (float)(wp - (double)g.wp_hi);
        rg.push_back(g);
        for (int64_t k = i; k < j; ++k) rec.push_back(h[k]);
        i = j;
      } else {
        rest.push_back(h[i]);
        ++i;
      }
    }
    gr = rg;
    ctx->rec_entries = (int64_t)rec.size();
    h = rec;
    h.insert(h.end(), rest.begin(), rest.end());
  }
  ctx->flist_d.reserve(sizeof(int32_t) * std::max<int64_t>(n, 1));
  ctx->groups_d.reserve(sizeof(FarGroup) * std::max<size_t>(gr.size(), 1));
  ctx->yacc.reserve(sizeof(double) * 6 * F * ne);
  if (n) BEM_CUDA(cudaMemcpyAsync(ctx->flist_d.p, h.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream));
  if (!gr.empty())
    BEM_CUDA(cudaMemcpyAsync(ctx->groups_d.p, gr.data(), sizeof(FarGroup) * gr.size(), cudaMemcpyHostToDevice,
                             ctx->stream));
  // zero the accumulator rows of the listed frequencies (contiguous runs in one memset each)
  std::vector<int32_t> sorted(h);
  std::sort(sorted.begin(), sorted.end());
  for (int64_t a = 0; a < n;) {
    int64_t b = a + 1;
    while (b < n && sorted[b] == sorted[b - 1] + 1) ++b;
    BEM_CUDA(cudaMemsetAsync(ctx->yacc.as<double>() + (int64_t)sorted[a] * ne * 6, 0,
                             sizeof(double) * 6 * ne * (b - a), ctx->stream));
    a = b;
  }
  return n;
}

// Resident CTAs per SM of an FP32 far-kernel instantiation (occupancy query, made once; the
// initialisation of a function-local static is thread-safe, and contexts on host threads of
// bem_solve_batch may launch concurrently).
template <int FT, bool REC>
static int far32_per_sm() {
  static const int n = [] {
    constexpr int TB = Cfg<float>::TB, S = Cfg<float>::S;
    const size_t smem = far_smem<float, TB, S, FT, false>();
    BEM_CUDA(cudaFuncSetAttribute(far32_kernel<TB, S, FT, REC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    int b = 0;
    BEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, far32_kernel<TB, S, FT, REC>, TB, smem));
    return std::max(b, 1);
  }();
  return n;
}

// Grid of a far-field launch: targets x CTA frequency groups x source splits, with the split
// chosen so that the grid covers `waves` waves of resident CTAs and no CTA sums more than
// `tiles` source tiles before its FP64 atomic add.
static int64_t far_split(int64_t ne, int64_t tb, int64_t groups, int S, int n_sm, int per_sm, int waves, int tiles,
                         int64_t* chunk_out) {
  const int64_t want = (int64_t)waves * n_sm * per_sm;
  int64_t nsplit = std::max<int64_t>(1, (want + tb * groups - 1) / (tb * groups));
  nsplit = std::max<int64_t>(nsplit, (ne + (int64_t)tiles * S - 1) / ((int64_t)tiles * S));
  nsplit = std::min<int64_t>(nsplit, 65535);
  int64_t chunk = (ne + nsplit - 1) / nsplit;
  chunk = ((chunk + S - 1) / S) * S;
  *chunk_out = chunk;
  return (ne + chunk - 1) / chunk;
}

template <int FT, bool REC>
static void launch_far32(bem_ctx* ctx, FarArgs<float>& a, int64_t ng, const FarShape& sh) {
  constexpr int TB = Cfg<float>::TB, S = Cfg<float>::S;
  const int64_t tb = grid_for(a.ne, TB), groups = REC ? ng : grid_for(a.nfl, FT);
  const int64_t nsplit = far_split(a.ne, tb, groups, S, ctx->n_sm > 0 ? ctx->n_sm : 152, far32_per_sm<FT, REC>(),
                                   sh.waves, sh.tiles, &a.chunk);
  const size_t smem = far_smem<float, TB, S, FT, false>();
  const dim3 grid((unsigned)tb, (unsigned)groups, (unsigned)nsplit);
  BEM_CUDA(cudaFuncSetAttribute(far32_kernel<TB, S, FT, REC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  far32_kernel<TB, S, FT, REC><<<grid, TB, smem, ctx->stream>>>(a);
}

// One far-field launch.  REC: over the group descriptors [g0, g0 + ng); else over the list
// entries [off, off + nfl), FT per CTA (FP32: the launch shape's ft).
template <class R, bool RESID, bool REC>
static void launch_far_part(bem_ctx* ctx, const cx<R>* x, int which, int64_t off, int64_t nfl, int64_t g0,
                            int64_t ng, const FarShape& sh) {
  constexpr int TB = Cfg<R>::TB, S = Cfg<R>::S, FT = Cfg<R>::FT;
  if (nfl <= 0) return;
  FarArgs<R> a;
  a.bcv = ctx->bc.set ? ctx->bc.d_value.as<double>() : nullptr;
  a.pfac = ctx->fs.pfac.as<cx<double>>();
  a.q4 = Geo<R>::q4(ctx);
  a.cen = Geo<R>::cen(ctx);
  a.nrm = Geo<R>::nrm(ctx);
  a.q4lo = ctx->mesh.q4_32lo.as<float4>();
  a.cenlo = ctx->mesh.c32lo.as<float4>();
  a.bc = ctx->bc.set ? ctx->bc.d_type.as<int8_t>() : nullptr;
  a.which = which;
  a.x = x;
  a.yacc = ctx->yacc.as<double>();
  a.fc = Geo<R>::fc(ctx);
  a.flist = ctx->flist_d.as<int32_t>() + off;
  a.groups = REC ? ctx->groups_d.as<FarGroup>() + g0 : nullptr;
  a.nfl = nfl;
  a.ne = ctx->mesh.ne;
  a.F = ctx->fs.F;
  a.m = Geo<R>::m(ctx);
  ProfScope ps(ctx, RESID ? PK_RES64 : (sizeof(R) == 4 ? PK_FAR32 : PK_FAR64), nfl);
  if constexpr (sizeof(R) == 4 && !RESID) {
    // the launch shape (frequencies per CTA, tiles per CTA, waves) from the tuning table
    switch (sh.ft) {
      case 1: launch_far32<1, REC>(ctx, a, ng, sh); break;
      case 4: launch_far32<4, REC>(ctx, a, ng, sh); break;
      case 8: launch_far32<8, REC>(ctx, a, ng, sh); break;
      default: launch_far32<12, REC>(ctx, a, ng, sh); break;
    }
  } else {
    // split the sources so that the grid covers about four waves of resident CTAs and a CTA
    // sums at most 2 source tiles before the FP64 atomic add
    const int64_t tb = grid_for(a.ne, TB), groups = REC ? ng : grid_for(nfl, FT);
    const int64_t nsplit = far_split(a.ne, tb, groups, S, ctx->n_sm > 0 ? ctx->n_sm : 152, Cfg<R>::kPerSM, 4, 2,
                                     &a.chunk);
    const size_t smem = far_smem<R, TB, S, FT, RESID>();
    const dim3 grid((unsigned)tb, (unsigned)groups, (unsigned)nsplit);
    BEM_CUDA(cudaFuncSetAttribute(far_kernel<R, TB, S, FT, RESID>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    far_kernel<R, TB, S, FT, RESID><<<grid, TB, smem, ctx->stream>>>(a);
  }
  BEM_LAUNCHED();
  ctx->launches++;
}

// Far field over the staged list: FP32 equally spaced runs (the leading rec_entries) by the
// recurrence kernel, the rest by the direct one.
template <class R, bool RESID>
static void launch_far(bem_ctx* ctx, const cx<R>* x, int which, int64_t nfl, const FarShape& sh = FarShape()) {
  const int64_t nrec = ctx->rec_entries;
  if constexpr (sizeof(R) == 4 && !RESID) {
    launch_far_part<R, RESID, true>(ctx, x, which, 0, nrec, 0, (int64_t)ctx->groups_h.size(), sh);
    launch_far_part<R, RESID, false>(ctx, x, which, nrec, nfl - nrec, 0, 0, sh);
  } else {
    launch_far_part<R, RESID, false>(ctx, x, which, 0, nfl, 0, 0, sh);
  }
}

template <class R>
static void launch_near(bem_ctx* ctx, const cx<R>* x, cx<R>* y, int which, int64_t nfl, bool resid) {
  NearArgs<R> a;
  a.resid = resid;
  a.bcv = ctx->bc.set ? ctx->bc.d_value.as<double>() : nullptr;
  a.pfac = ctx->fs.pfac.as<cx<double>>();
  a.q4 = Geo<R>::q4(ctx);
  a.q7 = Geo<R>::q7(ctx);
  a.cen = Geo<R>::cen(ctx);
  a.nrm = Geo<R>::nrm(ctx);
  a.ptr = ctx->mesh.near_ptr.as<int32_t>();
  a.col = ctx->mesh.near_col.as<int32_t>();
  a.bc = ctx->bc.set ? ctx->bc.d_type.as<int8_t>() : nullptr;
  a.which = which;
  a.Tself = ctx->fs.Tself.as<cx<double>>();
  a.Gself = ctx->fs.Gself.as<cx<double>>();
  a.x = x;
  a.y = y;
  a.yacc = ctx->yacc.as<double>();
  a.fc = Geo<R>::fc(ctx);
  a.flist = ctx->flist_d.as<int32_t>();
  a.nfl = nfl;
  a.ne = ctx->mesh.ne;
  a.F = ctx->fs.F;
  a.m = Geo<R>::m(ctx);
  ProfScope ps(ctx, sizeof(R) == 4 ? PK_NEAR32 : PK_NEAR64, nfl);
  // a warp per target when one thread per target would leave the SMs mostly idle
  const int64_t items = nfl * a.ne;
  if (items < (int64_t)4 * 128 * (ctx->n_sm > 0 ? ctx->n_sm : 152))
    near_kernel<R, true><<<grid_for(32 * items, 128), 128, 0, ctx->stream>>>(a);
  else
    near_kernel<R, false><<<grid_for(items, 128), 128, 0, ctx->stream>>>(a);
  BEM_LAUNCHED();
  ctx->launches++;
}

void apply_operator64(bem_ctx* ctx, const cx<double>* x, cx<double>* y, int which,
                      const std::vector<int32_t>* flist) {
  const int64_t n = stage_flist(ctx, flist, 0);
  if (!n) return;
  launch_far<double, false>(ctx, x, which, n);
  launch_near<double>(ctx, x, y, which, n, false);
  ctx->f64_applies++;
}

void near_residual64(bem_ctx* ctx, const cx<double>* x, cx<double>* r, int64_t nfl) {
  launch_near<double>(ctx, x, r, BEM_APPLY_A, nfl, true);
}

void residual64(bem_ctx* ctx, const cx<double>* x, cx<double>* r, const std::vector<int32_t>* flist) {
  BEM_REQUIRE(ctx->bc.set, "residual needs boundary conditions");
  const int64_t n = stage_flist(ctx, flist, 0);
  if (!n) return;
  launch_far<double, true>(ctx, x, BEM_APPLY_A, n);
  launch_near<double>(ctx, x, r, BEM_APPLY_A, n, true);
  ctx->f64_applies++;
}

void apply_operator32(bem_ctx* ctx, const cx<float>* x, cx<float>* y, int which,
                      const std::vector<int32_t>* flist) {
  if (which == BEM_APPLY_A && hm_active(ctx)) {
    // H-matrix far field (hmatrix.cu) in place of the direct far kernel
    const int64_t n = stage_flist(ctx, flist, 0);
    if (!n) return;
    hm_far32(ctx, x, n);
    launch_near<float>(ctx, x, y, which, n, false);
    ctx->f32_applies++;
    return;
  }
  const FarShape sh = far32_shape(ctx, flist ? (int64_t)flist->size() : ctx->fs.F);
  const int64_t n = stage_flist(ctx, flist, sh.ft);
  if (!n) return;
  launch_far<float, false>(ctx, x, which, n, sh);
  launch_near<float>(ctx, x, y, which, n, false);
  ctx->f32_applies++;
}

void apply_precond64(bem_ctx* ctx, const cx<double>* x, cx<double>* y, const int32_t* active) {
  const int64_t n = ctx->fs.F * ctx->mesh.ne;
  precond_kernel<double><<<grid_for(n, 128), 128, 0, ctx->stream>>>(
      ctx->fs.Minv64.as<cx<double>>(), x, y, active, ctx->mesh.ne, ctx->fs.F);
  BEM_LAUNCHED();
  ctx->launches++;
}

void apply_precond32(bem_ctx* ctx, const cx<float>* x, cx<float>* y, const int32_t* active) {
  const int64_t n = ctx->fs.F * ctx->mesh.ne;
  precond_kernel<float><<<grid_for(n, 128), 128, 0, ctx->stream>>>(
      ctx->fs.Minv32.as<cx<float>>(), x, y, active, ctx->mesh.ne, ctx->fs.F);
  BEM_LAUNCHED();
  ctx->launches++;
}

void known_data(bem_ctx* ctx, cx<double>* out) {
  const int64_t n = ctx->fs.F * ctx->mesh.ne * 3;
  known_data_kernel<<<grid_for(n, 256), 256, 0, ctx->stream>>>(
      ctx->fs.pfac.as<cx<double>>(), ctx->bc.d_value.as<double>(), out, ctx->mesh.ne, ctx->fs.F);
  BEM_LAUNCHED();
  ctx->launches++;
}

}  // namespace bem
