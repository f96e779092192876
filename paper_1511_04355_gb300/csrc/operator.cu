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
  const int8_t* bc;             // [ne] or null (all traction-given)
  int which;                    // BEM_APPLY_A / BEM_APPLY_K
  const cx<R>* x;               // [F][ne][3]
  cx<R>* y;                     // [F][ne][3]
  const FreqC<R>* fc;           // [F]
  const int32_t* active;        // [F] or null
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

template <class R, int TB, int S, int FT>
__global__ void __launch_bounds__(TB) far_kernel(const FarArgs<R> a) {
  using V = typename V4<R>::T;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  double* acc = reinterpret_cast<double*>(smem_raw);                 // [6 FT][TB]
  V* sq = reinterpret_cast<V*>(acc + 6 * FT * TB);                    // [S][4]
  V* sn = sq + 4 * S;                                                  // [S]
  cx<R>* sv = reinterpret_cast<cx<R>*>(sn + S);                       // [S][FT][4]
  FreqC<R>* sfc = reinterpret_cast<FreqC<R>*>(sv + 4 * FT * S);       // [FT]

  const int tid = threadIdx.x;
  const int64_t f0 = (int64_t)blockIdx.y * FT;
  const int nf = (int)min((int64_t)FT, a.F - f0);
  unsigned mask = 0;
  for (int k = 0; k < nf; ++k)
    if (!a.active || a.active[f0 + k]) mask |= 1u << k;
  if (mask == 0) return;
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
    if (tid < nf) sfc[tid] = a.fc[f0 + tid];
    else sfc[tid] = FreqC<R>{};
  }
#pragma unroll
  for (int k = 0; k < 6 * FT; ++k) acc[k * TB + tid] = 0.0;
  const MatC<R>& m = a.m;
  const R inv4pi = R(kInv4Pi);

  for (int64_t e0 = 0; e0 < a.ne; e0 += S) {
    const int ns = (int)min((int64_t)S, a.ne - e0);
    __syncthreads();
    for (int t = tid; t < 4 * ns; t += TB) sq[t] = a.q4[4 * e0 + t];
    for (int t = tid; t < ns; t += TB) {
      V n = a.nrm[e0 + t];
      n.w = (R)column_code(a.bc, e0 + t, a.which);
      sn[t] = n;
    }
    for (int t = tid; t < ns * FT; t += TB) {
      const int e = t / FT, k = t % FT;
      cx<R> v0 = mk(R(0), R(0)), v1 = v0, v2 = v0;
      if (k < nf) {
        const cx<R>* xv = a.x + ((f0 + k) * a.ne + e0 + e) * 3;
        v0 = xv[0];
        v1 = xv[1];
        v2 = xv[2];
      }
      const V n = a.nrm[e0 + e];
      cx<R>* o = sv + 4 * (e * FT + k);
      o[0] = v0;
      o[1] = v1;
      o[2] = v2;
      o[3] = mk(n.x * v0.r + n.y * v1.r + n.z * v2.r, n.x * v0.i + n.y * v1.i + n.z * v2.i);
    }
    __syncthreads();

    cx<R> part[FT][3];
#pragma unroll
    for (int k = 0; k < FT; ++k) part[k][0] = part[k][1] = part[k][2] = mk(R(0), R(0));

    for (int e = 0; e < ns; ++e) {
      const V nn = sn[e];
      const bool self = (e0 + e == i);
      const bool isU = fabs((float)nn.w) > 1.5f;
      const R sign = nn.w > 0 ? R(1) : R(-1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const V p = sq[4 * e + q];
        const R dx = p.x - xi0, dy = p.y - xi1, dz = p.z - xi2;
        const R r2 = self ? R(1) : dx * dx + dy * dy + dz * dz;
        const R rinv = rsqrt_r(r2);
        const R r = r2 * rinv;
        const R inv_r2 = rinv * rinv;
        const R rh0 = dx * rinv, rh1 = dy * rinv, rh2 = dz * rinv;
        const R w = self ? R(0) : p.w * sign;
        if (!isU) {
          const R drdn = rh0 * nn.x + rh1 * nn.y + rh2 * nn.z;
          const R cw = w * inv_r2 * inv4pi;
          const R cwd = cw * drdn;
#pragma unroll
          for (int k = 0; k < FT; ++k) {
            if (!((mask >> k) & 1u)) continue;
            const FreqC<R> fc = sfc[k];
            const cx<R>* v = sv + 4 * (e * FT + k);
            const cx<R> v0 = v[0], v1 = v[1], v2 = v[2], nv = v[3];
            const Radial<R> K = radial(r, inv_r2, fc, m);
            const TCoef<R> T = tcoef(K, m);
            const cx<R> rv = mk(rh0 * v0.r + rh1 * v1.r + rh2 * v2.r, rh0 * v0.i + rh1 * v1.i + rh2 * v2.i);
            const cx<R> t1 = cwd * T.A;
            const cx<R> t2 = (cw * T.A) * rv;
            const cx<R> t3 = cw * cfma(T.q1, nv, drdn * (T.q2 * rv));
            part[k][0] = cfma(t1, v0, axpy(nn.x, t2, axpy(rh0, t3, part[k][0])));
            part[k][1] = cfma(t1, v1, axpy(nn.y, t2, axpy(rh1, t3, part[k][1])));
            part[k][2] = cfma(t1, v2, axpy(nn.z, t2, axpy(rh2, t3, part[k][2])));
          }
        } else {
          const R cu = w * rinv * m.inv4pimu;
#pragma unroll
          for (int k = 0; k < FT; ++k) {
            if (!((mask >> k) & 1u)) continue;
            const FreqC<R> fc = sfc[k];
            const cx<R>* v = sv + 4 * (e * FT + k);
            const cx<R> v0 = v[0], v1 = v[1], v2 = v[2];
            const Radial<R> K = radial(r, inv_r2, fc, m);
            const cx<R> psi = cu * (K.Es - K.J);
            const cx<R> rv = mk(rh0 * v0.r + rh1 * v1.r + rh2 * v2.r, rh0 * v0.i + rh1 * v1.i + rh2 * v2.i);
            const cx<R> crv = (cu * axpy(R(-3), K.J, K.P)) * rv;
            part[k][0] = cfma(psi, v0, axpy(-rh0, crv, part[k][0]));
            part[k][1] = cfma(psi, v1, axpy(-rh1, crv, part[k][1]));
            part[k][2] = cfma(psi, v2, axpy(-rh2, crv, part[k][2]));
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < FT; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[(6 * k + 2 * c) * TB + tid] += (double)part[k][c].r;
        acc[(6 * k + 2 * c + 1) * TB + tid] += (double)part[k][c].i;
      }
  }
  if (!valid) return;
#pragma unroll
  for (int k = 0; k < FT; ++k) {
    if (!((mask >> k) & 1u)) continue;
    cx<R>* yo = a.y + ((f0 + k) * a.ne + i) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      yo[c] = mk((R)acc[(6 * k + 2 * c) * TB + tid], (R)acc[(6 * k + 2 * c + 1) * TB + tid]);
  }
}

template <class R, int TB, int S, int FT>
static size_t far_smem() {
  using V = typename V4<R>::T;
  return sizeof(double) * 6 * FT * TB + sizeof(V) * 5 * S + sizeof(cx<R>) * 4 * FT * S +
         sizeof(FreqC<R>) * FT;
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
  const cx<double>* Tself;  // [F][ne][9]
  const cx<double>* Gself;
  const cx<R>* x;
  cx<R>* y;
  const FreqC<R>* fc;
  const int32_t* active;
  int64_t ne, F;
  MatC<R> m;
};

template <class R>
__device__ __forceinline__ void add_point(R xi0, R xi1, R xi2, const typename V4<R>::T& p, R wsign,
                                          const typename V4<R>::T& nn, bool isU,
                                          const FreqC<R>& fc, const MatC<R>& m, const cx<R>* v,
                                          cx<R> nv, cx<R>* o) {
  const R dx = p.x - xi0, dy = p.y - xi1, dz = p.z - xi2;
  const R r2 = dx * dx + dy * dy + dz * dz;
  const R rinv = rsqrt_r(r2), r = r2 * rinv, inv_r2 = rinv * rinv;
  const R rh[3] = {dx * rinv, dy * rinv, dz * rinv};
  const Radial<R> K = radial(r, inv_r2, fc, m);
  const cx<R> rv = mk(rh[0] * v[0].r + rh[1] * v[1].r + rh[2] * v[2].r,
                      rh[0] * v[0].i + rh[1] * v[1].i + rh[2] * v[2].i);
  if (!isU) {
    const R drdn = rh[0] * nn.x + rh[1] * nn.y + rh[2] * nn.z;
    const R cw = p.w * wsign * inv_r2 * R(kInv4Pi);
    const TCoef<R> T = tcoef(K, m);
    const cx<R> t1 = (cw * drdn) * T.A;
    const cx<R> t2 = (cw * T.A) * rv;
    const cx<R> t3 = cw * cfma(T.q1, nv, drdn * (T.q2 * rv));
    const R nvec[3] = {nn.x, nn.y, nn.z};
    for (int c = 0; c < 3; ++c) o[c] = cfma(t1, v[c], axpy(nvec[c], t2, axpy(rh[c], t3, o[c])));
  } else {
    const R cu = p.w * wsign * rinv * m.inv4pimu;
    const cx<R> psi = cu * (K.Es - K.J);
    const cx<R> crv = (cu * axpy(R(-3), K.J, K.P)) * rv;
    for (int c = 0; c < 3; ++c) o[c] = cfma(psi, v[c], axpy(-rh[c], crv, o[c]));
  }
}

template <class R>
__global__ void near_kernel(const NearArgs<R> a) {
  using V = typename V4<R>::T;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= a.F * a.ne) return;
  const int64_t f = t / a.ne, i = t % a.ne;
  if (a.active && !a.active[f]) return;
  const V c = a.cen[i];
  const FreqC<R> fc = a.fc[f];
  cx<R> o[3] = {mk(R(0), R(0)), mk(R(0), R(0)), mk(R(0), R(0))};
  for (int32_t p = a.ptr[i]; p < a.ptr[i + 1]; ++p) {
    const int64_t e = a.col[p];
    const float code = column_code(a.bc, e, a.which);
    const bool isU = fabsf(code) > 1.5f;
    const R sign = code > 0 ? R(1) : R(-1);
    const V nn = a.nrm[e];
    const cx<R>* xv = a.x + (f * a.ne + e) * 3;
    const cx<R> v[3] = {xv[0], xv[1], xv[2]};
    const cx<R> nv = mk(nn.x * v[0].r + nn.y * v[1].r + nn.z * v[2].r,
                        nn.x * v[0].i + nn.y * v[1].i + nn.z * v[2].i);
    for (int q = 0; q < 7; ++q) add_point(c.x, c.y, c.z, a.q7[7 * e + q], sign, nn, isU, fc, a.m, v, nv, o);
    for (int q = 0; q < 4; ++q) add_point(c.x, c.y, c.z, a.q4[4 * e + q], -sign, nn, isU, fc, a.m, v, nv, o);
  }
  // own element: A_ii or K_ii from the FP64 singular blocks
  const int b = a.bc ? (int)a.bc[i] : 0;
  const bool useU = (b ^ a.which) != 0;
  const double sg = b ? -1.0 : 1.0;
  const cx<double>* blk = (useU ? a.Gself : a.Tself) + (f * a.ne + i) * 9;
  const cx<R>* xv = a.x + (f * a.ne + i) * 3;
  const cx<R> v[3] = {xv[0], xv[1], xv[2]};
  for (int r = 0; r < 3; ++r) {
    cx<R> s = mk(R(0), R(0));
    for (int cc = 0; cc < 3; ++cc) {
      cx<double> d = blk[3 * r + cc];
      if (!useU && r == cc) d.r += 0.5;
      s = cfma(mk((R)(sg * d.r), (R)(sg * d.i)), v[cc], s);
    }
    o[r] = o[r] + s;
  }
  cx<R>* yo = a.y + (f * a.ne + i) * 3;
  for (int r = 0; r < 3; ++r) yo[r] = yo[r] + o[r];
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
struct Cfg<float> {  // FP32: 128 targets x 8 frequencies per CTA, 64-element source tiles
  static constexpr int TB = 128, S = 64, FT = 8;
};
template <>
struct Cfg<double> {  // FP64: 128 targets x 4 frequencies per CTA, 32-element source tiles
  static constexpr int TB = 128, S = 32, FT = 4;
};

template <class R>
static void launch_far(bem_ctx* ctx, const cx<R>* x, cx<R>* y, int which, const int32_t* active) {
  constexpr int TB = Cfg<R>::TB, S = Cfg<R>::S, FT = Cfg<R>::FT;
  FarArgs<R> a;
  a.q4 = Geo<R>::q4(ctx);
  a.cen = Geo<R>::cen(ctx);
  a.nrm = Geo<R>::nrm(ctx);
  a.bc = ctx->bc.set ? ctx->bc.d_type.as<int8_t>() : nullptr;
  a.which = which;
  a.x = x;
  a.y = y;
  a.fc = Geo<R>::fc(ctx);
  a.active = active;
  a.ne = ctx->mesh.ne;
  a.F = ctx->fs.F;
  a.m = Geo<R>::m(ctx);
  const size_t smem = far_smem<R, TB, S, FT>();
  BEM_CUDA(cudaFuncSetAttribute(far_kernel<R, TB, S, FT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const dim3 grid(grid_for(a.ne, TB), grid_for(a.F, FT));
  ProfScope ps(ctx, sizeof(R) == 4 ? PK_FAR32 : PK_FAR64);
  far_kernel<R, TB, S, FT><<<grid, TB, smem, ctx->stream>>>(a);
  BEM_LAUNCHED();
  ctx->launches++;
}

template <class R>
static void launch_near(bem_ctx* ctx, const cx<R>* x, cx<R>* y, int which, const int32_t* active) {
  NearArgs<R> a;
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
  a.fc = Geo<R>::fc(ctx);
  a.active = active;
  a.ne = ctx->mesh.ne;
  a.F = ctx->fs.F;
  a.m = Geo<R>::m(ctx);
  ProfScope ps(ctx, sizeof(R) == 4 ? PK_NEAR32 : PK_NEAR64);
  near_kernel<R><<<grid_for(a.F * a.ne, 128), 128, 0, ctx->stream>>>(a);
  BEM_LAUNCHED();
  ctx->launches++;
}

void apply_operator64(bem_ctx* ctx, const cx<double>* x, cx<double>* y, int which,
                      const int32_t* active) {
  launch_far<double>(ctx, x, y, which, active);
  launch_near<double>(ctx, x, y, which, active);
  ctx->f64_applies++;
}

void apply_operator32(bem_ctx* ctx, const cx<float>* x, cx<float>* y, int which,
                      const int32_t* active) {
  launch_far<float>(ctx, x, y, which, active);
  launch_near<float>(ctx, x, y, which, active);
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
