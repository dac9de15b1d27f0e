// Batched vector kernels of the solver (see hx_vec.cuh).
#include "hx_complex.cuh"
#include "hx_internal.h"
#include "hx_launch.cuh"
#include "hx_vec.cuh"

namespace hx {
namespace {

constexpr int kThreads = 256;

inline dim3 grid_for(long long N, int R, int per_thread = 4) {
  long long b = (N + (long long)kThreads * per_thread - 1) / ((long long)kThreads * per_thread);
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return dim3((unsigned)b, (unsigned)R);
}

template <class C> __device__ __forceinline__ C from_d2(double2 a);
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }

// block-wide sum of a double2 (all threads get the result in lane 0 of warp 0)
__device__ double2 block_sum(double2 v) {
  __shared__ double2 sh[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  if (w == 0) {
    if (l < kThreads / 32) t = sh[l];
    for (int o = 16; o > 0; o >>= 1) {
      t.x += __shfl_down_sync(0xffffffffu, t.x, o);
      t.y += __shfl_down_sync(0xffffffffu, t.y, o);
    }
  }
  return t;
}

template <typename T, bool NORM>
__global__ void __launch_bounds__(kThreads)
dot_partial(const typename CT<T>::type* __restrict__ a, const typename CT<T>::type* __restrict__ b,
            long long N, double2* __restrict__ part) {
  pdl_enter();
  using C = typename CT<T>::type;
  const int r = blockIdx.y;
  const C* ar = a + (long long)r * N;
  const C* br = b + (long long)r * N;
  T sx = 0, sy = 0;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < N;
       i += (long long)gridDim.x * kThreads) {
    const C u = ar[i];
    if (NORM) {
      sx = fma(u.x, u.x, fma(u.y, u.y, sx));
    } else {
      const C w = br[i];
      sx = fma(u.x, w.x, fma(u.y, w.y, sx));     // Re(conj(u) w)
      sy = fma(u.x, w.y, fma(-u.y, w.x, sy));    // Im(conj(u) w)
    }
  }
  const double2 t = block_sum(make_double2((double)sx, (double)sy));
  if (threadIdx.x == 0) part[(long long)r * gridDim.x + blockIdx.x] = t;
}

__global__ void __launch_bounds__(kThreads)
dot_finish(const double2* __restrict__ part, int nblk, double2* out, double* out_re) {
  pdl_enter();
  const int r = blockIdx.x;
  double2 s = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < nblk; i += kThreads) {
    const double2 p = part[(long long)r * nblk + i];
    s.x += p.x;
    s.y += p.y;
  }
  const double2 t = block_sum(s);
  if (threadIdx.x == 0) {
    if (out) out[r] = t;
    if (out_re) out_re[r] = t.x;
  }
}

template <typename T>
__global__ void bicg_p_k(typename CT<T>::type* __restrict__ p, const typename CT<T>::type* __restrict__ r,
                         const typename CT<T>::type* __restrict__ v, const double2* beta,
                         const double2* omega, long long N) {
  pdl_enter();
  using C = typename CT<T>::type;
  const int k = blockIdx.y;
  const C be = from_d2<C>(beta[k]), om = from_d2<C>(omega[k]);
  const long long o = (long long)k * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const C pv = p[o + i], vv = v[o + i];
    const C t = csub(pv, cmul(om, vv));
    p[o + i] = cfma(be, t, r[o + i]);
  }
}

template <typename T>
__global__ void bicg_s_k(typename CT<T>::type* __restrict__ sv, const typename CT<T>::type* __restrict__ r,
                         const typename CT<T>::type* __restrict__ v, const double2* alpha, long long N) {
  pdl_enter();
  using C = typename CT<T>::type;
  const int k = blockIdx.y;
  const C al = from_d2<C>(alpha[k]);
  const C mal = cmk(-al.x, -al.y);
  const long long o = (long long)k * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    sv[o + i] = cfma(mal, v[o + i], r[o + i]);
}

// full weighting: coarse node I <- fine nodes 2I + s, s in {-1,0,1}^3, weight
// prod_d (1/2)^{|s_d|} / 8; fine nodes outside the grid are zero.
// fp: x-row pitch of the fine field (elements, >= fx).
template <typename T>
__global__ void restrict_k(const typename CT<T>::type* __restrict__ f, int fx, int fy, int fz, long long fp,
                           typename CT<T>::type* __restrict__ c, int cx, int cy, int cz) {
  pdl_enter();
  using C = typename CT<T>::type;
  const long long Nc = (long long)cx * cy * cz, Nf = fp * fy * fz;
  const int r = blockIdx.y;
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < Nc;
       I += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(I % cx), Y = (int)((I / cx) % cy), Z = (int)(I / ((long long)cx * cy));
    C acc = czero<C>();
    for (int sz = -1; sz <= 1; ++sz) {
      const int z = 2 * Z + sz;
      if (z < 0 || z >= fz) continue;
      for (int sy = -1; sy <= 1; ++sy) {
        const int y = 2 * Y + sy;
        if (y < 0 || y >= fy) continue;
        for (int sx = -1; sx <= 1; ++sx) {
          const int x = 2 * X + sx;
          if (x < 0 || x >= fx) continue;
          const T w = (T)1 / (T)(8 << (abs(sx) + abs(sy) + abs(sz)));
          acc = cfmar(w, f[(long long)r * Nf + ((long long)z * fy + y) * fp + x], acc);
        }
      }
    }
    c[(long long)r * Nc + I] = acc;
  }
}

// trilinear prolongation added to the fine field
// fp: x-row pitch of the fine field (elements, >= fx); padding is not written.
template <typename T>
__global__ void prolong_k(typename CT<T>::type* __restrict__ f, int fx, int fy, int fz, long long fp,
                          const typename CT<T>::type* __restrict__ c, int cx, int cy, int cz) {
  pdl_enter();
  using C = typename CT<T>::type;
  const long long Nc = (long long)cx * cy * cz, Nf = (long long)fx * fy * fz, Nfp = fp * fy * fz;
  const int r = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Nf;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % fx), y = (int)((i / fx) % fy), z = (int)(i / ((long long)fx * fy));
    const long long fi = ((long long)z * fy + y) * fp + x;
    int ix[2], iy[2], iz[2];
    T wx[2], wy[2], wz[2];
    auto split = [](int p, int nc, int* id, T* w) {
      if ((p & 1) == 0) { id[0] = p / 2; w[0] = 1; id[1] = 0; w[1] = 0; }
      else {
        id[0] = p / 2; w[0] = (T)0.5;
        id[1] = p / 2 + 1; w[1] = p / 2 + 1 < nc ? (T)0.5 : (T)0;
        if (id[1] >= nc) id[1] = nc - 1;
      }
    };
    split(x, cx, ix, wx);
    split(y, cy, iy, wy);
    split(z, cz, iz, wz);
    C acc = czero<C>();
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int d = 0; d < 2; ++d) {
          const T w = wz[a] * wy[b] * wx[d];
          if (w != (T)0)
            acc = cfmar(w, c[(long long)r * Nc + ((long long)iz[a] * cy + iy[b]) * cx + ix[d]], acc);
        }
    f[(long long)r * Nfp + fi] = cadd(f[(long long)r * Nfp + fi], acc);
  }
}

__global__ void inject_v_k(const float* __restrict__ vf, int fx, int fy, float* __restrict__ vc,
                           int cx, int cy, int cz) {
  pdl_enter();
  const long long Nc = (long long)cx * cy * cz;
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < Nc;
       I += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(I % cx), Y = (int)((I / cx) % cy), Z = (int)(I / ((long long)cx * cy));
    vc[I] = vf[((long long)(2 * Z) * fy + 2 * Y) * fx + 2 * X];
  }
}

// Coarse velocity from the full-weighting average (1/4, 1/2, 1/4 per axis,
// renormalised at the grid's faces) of the slowness squared 1/v^2 around the
// fine node 2X: the coefficient of the mass term, so a coarse node sees the
// bodies its neighbourhood holds instead of one sample of them.
__global__ void coarsen_slowness_k(const float* __restrict__ vf, int fx, int fy, int fz, float* __restrict__ vc,
                                   int cx, int cy, int cz) {
  pdl_enter();
  const long long Nc = (long long)cx * cy * cz;
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < Nc;
       I += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(I % cx), Y = (int)((I / cx) % cy), Z = (int)(I / ((long long)cx * cy));
    float acc = 0.f, wsum = 0.f;
    for (int dz = -1; dz <= 1; ++dz) {
      const int z = 2 * Z + dz;
      if (z < 0 || z >= fz) continue;
      const float wz = dz == 0 ? 0.5f : 0.25f;
      for (int dy = -1; dy <= 1; ++dy) {
        const int y = 2 * Y + dy;
        if (y < 0 || y >= fy) continue;
        const float wy = wz * (dy == 0 ? 0.5f : 0.25f);
        const float* row = vf + ((long long)z * fy + y) * fx;
        for (int dx = -1; dx <= 1; ++dx) {
          const int x = 2 * X + dx;
          if (x < 0 || x >= fx) continue;
          const float w = wy * (dx == 0 ? 0.5f : 0.25f);
          const float sl = 1.f / row[x];
          acc = fmaf(w, sl * sl, acc);
          wsum += w;
        }
      }
    }
    vc[I] = rsqrtf(acc / wsum);
  }
}

// The complex64 side may use a padded x-row pitch p32 (rows of nx points);
// the complex128 side is unpadded.  Padding is neither read nor written.
__global__ void cast_scale_k(const double2* __restrict__ r64, float2* __restrict__ r32,
                             const double* scale, long long N, int nx, long long p32) {
  pdl_enter();
  const int k = blockIdx.y;
  const double s = scale[k];
  const long long o = (long long)k * N, o32 = (long long)k * (N / nx) * p32;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 a = r64[o + i];
    const long long row = i / nx;
    r32[o32 + row * p32 + (i - row * nx)] = make_float2((float)(a.x * s), (float)(a.y * s));
  }
}

template <class D>
__global__ void axpy_mixed_k(double2* __restrict__ x, const D* __restrict__ d,
                             const double* scale, long long N, int nx, long long pd) {
  pdl_enter();
  const int k = blockIdx.y;
  const double s = scale[k];
  const long long o = (long long)k * N, od = (long long)k * (N / nx) * pd;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / nx;
    const D a = d[od + row * pd + (i - row * nx)];
    double2 v = x[o + i];
    v.x = fma(s, (double)a.x, v.x);
    v.y = fma(s, (double)a.y, v.y);
    x[o + i] = v;
  }
}

template <typename T>
__global__ void add_sources_k(typename CT<T>::type* r, long long N, const SourceEntry* e, int n) {
  pdl_enter();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    T* p = (T*)(r + (long long)e[k].rhs * N + e[k].idx);
    atomicAdd(p, (T)e[k].re);
    atomicAdd(p + 1, (T)e[k].im);
  }
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ bool tiny(double2 a) { return !(a.x * a.x + a.y * a.y > 1e-300); }

// Per-RHS scalar steps of BiCGStab (thread 0 of the last block of RHS r).
__device__ void beta_step(const BicgScalars& sc, int r) {
  if (!sc.active[r]) { sc.beta[r] = make_double2(0, 0); return; }
  if (tiny(sc.rho[r]) || tiny(sc.omega[r])) { sc.beta[r] = make_double2(0, 0); sc.brk[r] = 1; return; }
  sc.beta[r] = cdiv(cmul(sc.rho_new[r], sc.alpha[r]), cmul(sc.rho[r], sc.omega[r]));
  sc.rho[r] = sc.rho_new[r];
}

__device__ void alpha_step(const BicgScalars& sc, int r) {
  if (!sc.active[r]) { sc.alpha[r] = make_double2(0, 0); return; }
  if (tiny(sc.rv[r])) { sc.alpha[r] = make_double2(0, 0); sc.active[r] = 0; sc.brk[r] = 1; return; }
  sc.alpha[r] = cdiv(sc.rho[r], sc.rv[r]);
}

// omega = (t, s) / (t, t); with the safeguard kappa > 0, where the cosine
// |(t, s)| / (|t| |s|) is below kappa omega is scaled by kappa / cosine
// (Sleijpen and van der Vorst 1995).  ss = (s, s).
__device__ void omega_step(const BicgScalars& sc, int r, double ss) {
  if (!sc.active[r]) { sc.omega[r] = make_double2(0, 0); return; }
  if (!(sc.tt[r] > 1e-300)) { sc.omega[r] = make_double2(0, 0); sc.active[r] = 0; sc.brk[r] = 1; return; }
  double2 om = make_double2(sc.ts[r].x / sc.tt[r], sc.ts[r].y / sc.tt[r]);
  if (sc.kappa > 0 && ss > 1e-300) {
    const double cs = sqrt(sc.ts[r].x * sc.ts[r].x + sc.ts[r].y * sc.ts[r].y) / sqrt(sc.tt[r] * ss);
    if (cs < sc.kappa && cs > 0) {
      const double g = sc.kappa / cs;
      om = make_double2(om.x * g, om.y * g);
    }
  }
  sc.omega[r] = om;
}

// sum of nblk partials in block order (the same order as dot_finish)
__device__ double2 partials_sum(const double2* p, int nblk) {
  double2 s = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < nblk; i += kThreads) {
    const double2 v = __ldcg(p + i);
    s.x += v.x;
    s.y += v.y;
  }
  return block_sum(s);
}

// The end of a one-launch reduction: block b's sums t (and q) become
// partials; the last block of RHS r to arrive adds the partials in block
// order, stores the result and takes the scalar step.  Call with the block's
// sums in thread 0 (block_sum), from every thread of the block.
template <int KIND>
__device__ void reduce_tail(double2 t, double2 q, double2* part, const BicgScalars& sc) {
  constexpr bool TWO = KIND == kRedOmega || KIND == kRedBetaNorm;
  const int r = blockIdx.y, nb = gridDim.x;
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    part[(long long)r * nb + blockIdx.x] = t;
    if (TWO) part[(long long)(gridDim.y + r) * nb + blockIdx.x] = q;
    __threadfence();                                   // partials visible before the arrival
    s_last = atomicAdd(sc.count + r, 1u) == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double2 f = partials_sum(part + (long long)r * nb, nb);
  double2 g = make_double2(0.0, 0.0);
  if (TWO) g = partials_sum(part + (long long)(gridDim.y + r) * nb, nb);
  if (threadIdx.x == 0) {
    sc.count[r] = 0;
    if (KIND == kRedBeta || KIND == kRedBetaNorm) { sc.rho_new[r] = f; beta_step(sc, r); }
    if (KIND == kRedAlpha) { sc.rv[r] = f; alpha_step(sc, r); }
    if (KIND == kRedOmega) { sc.ts[r] = f; sc.tt[r] = g.x; omega_step(sc, r, g.y); }
    if (KIND == kRedNorm) sc.rn2[r] = f.x;
    if (KIND == kRedBetaNorm) sc.rn2[r] = g.x;
  }
}

// One-launch reduction + scalar step (see launch_bicg_reduce).  The per-thread
// and per-block arithmetic is that of dot_partial / dot_finish.
template <typename T, int KIND>
__global__ void __launch_bounds__(kThreads)
bicg_reduce_k(const typename CT<T>::type* __restrict__ a, const typename CT<T>::type* __restrict__ b,
              long long N, double2* __restrict__ part, BicgScalars sc) {
  pdl_enter();
  using C = typename CT<T>::type;
  const int r = blockIdx.y;
  const C* ar = a + (long long)r * N;
  const C* br = b + (long long)r * N;
  T sx = 0, sy = 0, qx = 0, qy = 0;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < N;
       i += (long long)gridDim.x * kThreads) {
    const C u = ar[i];
    if (KIND == kRedNorm) {
      sx = fma(u.x, u.x, fma(u.y, u.y, sx));
    } else {
      const C w = br[i];
      sx = fma(u.x, w.x, fma(u.y, w.y, sx));     // Re(conj(u) w)
      sy = fma(u.x, w.y, fma(-u.y, w.x, sy));    // Im(conj(u) w)
      if (KIND == kRedOmega) {
        qx = fma(u.x, u.x, fma(u.y, u.y, qx));   // (t, t)
        qy = fma(w.x, w.x, fma(w.y, w.y, qy));   // (s, s)
      }
    }
  }
  const double2 t = block_sum(make_double2((double)sx, (double)sy));
  double2 q = make_double2(0.0, 0.0);
  if (KIND == kRedOmega) q = block_sum(make_double2((double)qx, (double)qy));
  reduce_tail<KIND>(t, q, part, sc);
}

// x += alpha phat + omega shat;  r = s - omega t;  then the kRedBetaNorm
// reduction of the new r: rho_new = (rhat, r), the beta step of the next
// iteration, rn2 = |r|^2.  Same block partition as bicg_reduce_k, so the
// sums are those of the separate reductions.
template <typename T>
__global__ void __launch_bounds__(kThreads)
bicg_xr_reduce_k(typename CT<T>::type* __restrict__ x, typename CT<T>::type* __restrict__ r,
                 const typename CT<T>::type* __restrict__ sv, const typename CT<T>::type* __restrict__ ph,
                 const typename CT<T>::type* __restrict__ sh, const typename CT<T>::type* __restrict__ t,
                 const typename CT<T>::type* __restrict__ rhat, long long N, double2* __restrict__ part,
                 BicgScalars sc) {
  pdl_enter();
  using C = typename CT<T>::type;
  const int k = blockIdx.y;
  const C al = from_d2<C>(sc.alpha[k]), om = from_d2<C>(sc.omega[k]);
  const C mom = cmk(-om.x, -om.y);
  const long long o = (long long)k * N;
  T sx = 0, sy = 0, qx = 0;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < N;
       i += (long long)gridDim.x * kThreads) {
    x[o + i] = cfma(om, sh[o + i], cfma(al, ph[o + i], x[o + i]));
    const C w = cfma(mom, t[o + i], sv[o + i]);
    r[o + i] = w;
    const C u = rhat[o + i];
    sx = fma(u.x, w.x, fma(u.y, w.y, sx));
    sy = fma(u.x, w.y, fma(-u.y, w.x, sy));
    qx = fma(w.x, w.x, fma(w.y, w.y, qx));
  }
  const double2 tt = block_sum(make_double2((double)sx, (double)sy));
  const double2 q = block_sum(make_double2((double)qx, 0.0));
  reduce_tail<kRedBetaNorm>(tt, q, part, sc);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
dense_matvec_k(const typename CT<T>::type* __restrict__ M, const typename CT<T>::type* __restrict__ b,
               typename CT<T>::type* __restrict__ out, long long n) {
  pdl_enter();
  using C = typename CT<T>::type;
  const long long i = blockIdx.x;
  const int r = blockIdx.y;
  const C* row = M + i * n;
  const C* br = b + (long long)r * n;
  double sx = 0, sy = 0;
  for (long long j = threadIdx.x; j < n; j += kThreads) {
    const C a = row[j], x = br[j];
    sx += (double)a.x * x.x - (double)a.y * x.y;
    sy += (double)a.x * x.y + (double)a.y * x.x;
  }
  const double2 t = block_sum(make_double2(sx, sy));
  if (threadIdx.x == 0) out[(long long)r * n + i] = from_d2<C>(t);
}

}  // namespace

template <typename T>
cudaError_t launch_dense_matvec(const void* M, const void* b, void* out, long long n, int R,
                                cudaStream_t s) {
  using C = typename CT<T>::type;
  (void)launch_k(dense_matvec_k<T>, dim3((unsigned)n, R), kThreads, 0, s, (const C*)M, (const C*)b, (C*)out, n);
  count_launch(1);
  return cudaGetLastError();
}
template cudaError_t launch_dense_matvec<float>(const void*, const void*, void*, long long, int, cudaStream_t);
template cudaError_t launch_dense_matvec<double>(const void*, const void*, void*, long long, int, cudaStream_t);

int reduce_blocks(long long N) {
  long long b = (N + 1023) / 1024;
  if (b < 1) b = 1;
  if (b > 2048) b = 2048;
  return (int)b;
}

template <typename T>
cudaError_t launch_norm2(const void* a, long long N, int R, double2* part, double* out, cudaStream_t s) {
  using C = typename CT<T>::type;
  const int nb = reduce_blocks(N);
  (void)launch_k(dot_partial<T, true>, dim3(nb, R), kThreads, 0, s, (const C*)a, (const C*)a, N, part);
  (void)launch_k(dot_finish, R, kThreads, 0, s, part, nb, nullptr, out);
  count_launch(2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bicg_p(void* p, const void* r, const void* v, const double2* beta,
                          const double2* omega, long long N, int R, cudaStream_t s) {
  using C = typename CT<T>::type;
  (void)launch_k(bicg_p_k<T>, grid_for(N, R), kThreads, 0, s, (C*)p, (const C*)r, (const C*)v, beta, omega, N);
  count_launch(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bicg_s(void* sv, const void* r, const void* v, const double2* alpha, long long N,
                          int R, cudaStream_t s) {
  using C = typename CT<T>::type;
  (void)launch_k(bicg_s_k<T>, grid_for(N, R), kThreads, 0, s, (C*)sv, (const C*)r, (const C*)v, alpha, N);
  count_launch(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const void* fine, const int nf[3], void* coarse, const int nc[3], int R,
                            cudaStream_t s, long long fpitch) {
  using C = typename CT<T>::type;
  const long long Nc = (long long)nc[0] * nc[1] * nc[2];
  (void)launch_k(restrict_k<T>, grid_for(Nc, R, 1), kThreads, 0, s, (const C*)fine, nf[0], nf[1], nf[2],
                 fpitch > 0 ? fpitch : (long long)nf[0], (C*)coarse, nc[0], nc[1], nc[2]);
  count_launch(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(void* fine, const int nf[3], const void* coarse, const int nc[3], int R,
                               cudaStream_t s, long long fpitch) {
  using C = typename CT<T>::type;
  const long long Nf = (long long)nf[0] * nf[1] * nf[2];
  (void)launch_k(prolong_k<T>, grid_for(Nf, R, 1), kThreads, 0, s, (C*)fine, nf[0], nf[1], nf[2],
                 fpitch > 0 ? fpitch : (long long)nf[0], (const C*)coarse, nc[0], nc[1], nc[2]);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_velocity(const float* vf, const int nf[3], float* vc, const int nc[3], int mode,
                                   cudaStream_t s) {
  const long long Nc = (long long)nc[0] * nc[1] * nc[2];
  if (mode == 1)
    (void)launch_k(coarsen_slowness_k, grid_for(Nc, 1, 1), kThreads, 0, s, vf, nf[0], nf[1], nf[2], vc, nc[0],
                   nc[1], nc[2]);
  else
    (void)launch_k(inject_v_k, grid_for(Nc, 1, 1), kThreads, 0, s, vf, nf[0], nf[1], vc, nc[0], nc[1], nc[2]);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_cast_scale(const double2* r64, float2* r32, const double* scale, long long N, int R,
                              cudaStream_t s, int nx, long long p32) {
  (void)launch_k(cast_scale_k, grid_for(N, R), kThreads, 0, s, r64, r32, scale, N, nx, p32 > 0 ? p32 : (long long)nx);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_axpy_mixed(double2* x64, const float2* d32, const double* scale, long long N, int R,
                              cudaStream_t s, int nx, long long p32) {
  (void)launch_k(axpy_mixed_k<float2>, grid_for(N, R), kThreads, 0, s, x64, d32, scale, N, nx,
                 p32 > 0 ? p32 : (long long)nx);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_axpy_c128(double2* x64, const double2* d64, const double* scale, long long N, int R,
                             cudaStream_t s) {
  (void)launch_k(axpy_mixed_k<double2>, grid_for(N, R), kThreads, 0, s, x64, d64, scale, N, 1, 1LL);
  count_launch(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copy(void* y, const void* x, long long n, cudaStream_t s) {
  return cudaMemcpyAsync(y, x, n * 2 * sizeof(T), cudaMemcpyDeviceToDevice, s);
}

template <typename T>
cudaError_t launch_add_sources(void* r, long long N, const SourceEntry* e, int n, cudaStream_t s) {
  using C = typename CT<T>::type;
  if (n <= 0) return cudaSuccess;
  (void)launch_k(add_sources_k<T>, (n + 127) / 128, 128, 0, s, (C*)r, N, e, n);
  count_launch(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bicg_reduce(int kind, const void* a, const void* b, long long N, int R, double2* part,
                               const BicgScalars& sc, cudaStream_t s) {
  using C = typename CT<T>::type;
  const dim3 g(reduce_blocks(N), R);
  const C *ca = (const C*)a, *cb = (const C*)(b ? b : a);
  switch (kind) {
    case kRedBeta: (void)launch_k(bicg_reduce_k<T, kRedBeta>, g, kThreads, 0, s, ca, cb, N, part, sc); break;
    case kRedAlpha: (void)launch_k(bicg_reduce_k<T, kRedAlpha>, g, kThreads, 0, s, ca, cb, N, part, sc); break;
    case kRedOmega: (void)launch_k(bicg_reduce_k<T, kRedOmega>, g, kThreads, 0, s, ca, cb, N, part, sc); break;
    case kRedNorm: (void)launch_k(bicg_reduce_k<T, kRedNorm>, g, kThreads, 0, s, ca, cb, N, part, sc); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bicg_xr_reduce(void* x, void* r, const void* sv, const void* phat, const void* shat,
                                  const void* t, const void* rhat, long long N, int R, double2* part,
                                  const BicgScalars& sc, cudaStream_t s) {
  using C = typename CT<T>::type;
  (void)launch_k(bicg_xr_reduce_k<T>, dim3(reduce_blocks(N), R), kThreads, 0, s, (C*)x, (C*)r, (const C*)sv,
                 (const C*)phat, (const C*)shat, (const C*)t, (const C*)rhat, N, part, sc);
  count_launch(1);
  return cudaGetLastError();
}

#define HX_INST(T)                                                                                  \
  template cudaError_t launch_bicg_reduce<T>(int, const void*, const void*, long long, int, double2*, \
                                             const BicgScalars&, cudaStream_t);                   \
  template cudaError_t launch_bicg_xr_reduce<T>(void*, void*, const void*, const void*, const void*, \
                                                const void*, const void*, long long, int, double2*, \
                                                const BicgScalars&, cudaStream_t);                \
  template cudaError_t launch_norm2<T>(const void*, long long, int, double2*, double*,             \
                                       cudaStream_t);                                              \
  template cudaError_t launch_bicg_p<T>(void*, const void*, const void*, const double2*,           \
                                        const double2*, long long, int, cudaStream_t);             \
  template cudaError_t launch_bicg_s<T>(void*, const void*, const void*, const double2*,           \
                                        long long, int, cudaStream_t);                             \
  template cudaError_t launch_restrict<T>(const void*, const int*, void*, const int*, int,         \
                                          cudaStream_t, long long);                                \
  template cudaError_t launch_prolong_add<T>(void*, const int*, const void*, const int*, int,      \
                                             cudaStream_t, long long);                                        \
  template cudaError_t launch_copy<T>(void*, const void*, long long, cudaStream_t);                \
  template cudaError_t launch_add_sources<T>(void*, long long, const SourceEntry*, int,            \
                                             cudaStream_t);
HX_INST(float)
HX_INST(double)

}  // namespace hx
