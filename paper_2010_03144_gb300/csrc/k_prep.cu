// K1: prediction preparation and input checksums (the first two loops of Algorithm 1 of the
// paper: regression, checksums, sampling).
//
// One thread per block, a warp per 32 consecutive blocks. A single pass over the block
// computes, from the input as it is when compression starts:
//   * sum_in / isum_in over the block's 32-bit words (Algorithm 1; Sec. 3.2, 5.4),
//   * the regression sums (per row first, then per block) and the closed-form least-squares
//     coefficients,
//   * the Lorenzo estimate E_lor on the original values of the sample rows,
//   * the value range for the value-range relative bound;
// the regression estimate E_reg, which needs the coefficients, is taken by K2 just before it
// predicts the block (its re-read of the block then hits the cache).
// Full blocks of the common shapes take a fast path with compile-time edges; edge blocks and
// other shapes take the generic path. A one-thread kernel then turns the range into eb.
#include <algorithm>
#include <type_traits>

#include "sdcsz_internal.cuh"

namespace sdcsz {

namespace {

template <typename T>
__device__ __forceinline__ void mad_wide(unsigned long long& acc, uint32_t a, uint32_t b) {
  asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

template <typename T>
__device__ __forceinline__ void cks(T v, uint32_t k, unsigned long long& sum, unsigned long long& isum) {
  const uint32_t w0 = FT<T>::lo(v);
  if (FT<T>::W == 1) {
    mad_wide<T>(sum, w0, 1u);
    mad_wide<T>(isum, w0, k + 1);
  } else {
    const uint32_t w1 = FT<T>::hi(v);
    mad_wide<T>(sum, w0, 1u);
    mad_wide<T>(sum, w1, 1u);
    mad_wide<T>(isum, w0, 2 * k + 1);
    mad_wide<T>(isum, w1, 2 * k + 2);
  }
}

template <typename T>
__device__ __forceinline__ void minmax(T v, T& mn, T& mx) {
  if (FT<T>::finite(v)) {
    mn = v < mn ? v : mn;
    mx = v > mx ? v : mx;
  }
}

__device__ __forceinline__ float denom(uint32_t P, uint32_t ed) {
  return __double2float_rn(__ddiv_rn(__dmul_rn((double)P, __dsub_rn(__dmul_rn((double)ed, (double)ed), 1.0)), 12.0));
}

// The same denominator for a block shape known at compile time. P (e^2 - 1) / 12 is an integer
// below 2^24 for every compile-time shape (cubes 4..16, squares 8..16), so the double
// arithmetic is exact and the value equals denom's bit for bit.
__host__ __device__ constexpr float denom_c(uint32_t P, uint32_t ed) {
  return (float)((double)P * ((double)ed * (double)ed - 1.0) / 12.0);
}

// Coefficients from the block sums (slopes of the active axes, then the intercept); D[a] is
// the denominator of axis a (denom of its extent), used only where the extent exceeds 1.
template <int NDIM>
__device__ __forceinline__ bool coefficients(uint32_t P, const uint32_t e[3], const float D[3], float S0, float Si,
                                             float Sj, float Sl, float c0, float c1, float c2, float cf[4]) {
  const float mean = __fdiv_rn(S0, (float)P);
  if (NDIM == 3) {
    cf[0] = e[0] > 1 ? __fdiv_rn(Si, D[0]) : 0.0f;
    cf[1] = e[1] > 1 ? __fdiv_rn(Sj, D[1]) : 0.0f;
    cf[2] = e[2] > 1 ? __fdiv_rn(Sl, D[2]) : 0.0f;
    float acc = __fmul_rn(cf[0], c0);
    acc = __fadd_rn(acc, __fmul_rn(cf[1], c1));
    acc = __fadd_rn(acc, __fmul_rn(cf[2], c2));
    cf[3] = __fsub_rn(mean, acc);
  } else if (NDIM == 2) {
    cf[0] = e[1] > 1 ? __fdiv_rn(Sj, D[1]) : 0.0f;
    cf[1] = e[2] > 1 ? __fdiv_rn(Sl, D[2]) : 0.0f;
    float acc = __fmul_rn(cf[0], c1);
    acc = __fadd_rn(acc, __fmul_rn(cf[1], c2));
    cf[2] = __fsub_rn(mean, acc);
    cf[3] = 0.0f;
  } else {
    cf[0] = e[2] > 1 ? __fdiv_rn(Sl, D[2]) : 0.0f;
    cf[1] = __fsub_rn(mean, __fmul_rn(cf[0], c2));
    cf[2] = cf[3] = 0.0f;
  }
  bool finite = true;
  for (int a = 0; a <= NDIM; ++a) finite = finite && isfinite(cf[a]);
  return finite;
}

// Range reduction to the grid-wide minimum/maximum keys.
template <typename T>
__device__ __forceinline__ void reduce_range(T mn, T mx, State* st) {
  __shared__ unsigned long long s_min[32], s_max[32];
  unsigned long long kmin_inv = (mn <= mx) ? ~FT<T>::key(mn) : 0ull;
  unsigned long long kmax = (mn <= mx) ? FT<T>::key(mx) : 0ull;
  for (int o = 16; o > 0; o >>= 1) {
    kmin_inv = max(kmin_inv, __shfl_xor_sync(0xffffffffu, kmin_inv, o));
    kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    s_min[threadIdx.x >> 5] = kmin_inv;
    s_max[threadIdx.x >> 5] = kmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, m = 0;
    for (uint32_t q = 0; q < (blockDim.x + 31) / 32; ++q) {
      a = max(a, s_min[q]);
      m = max(m, s_max[q]);
    }
    if (m) {
      atomicMax(&st->min_key, a);
      atomicMax(&st->max_key, m);
    }
  }
}

template <typename T, int B2>
__device__ __forceinline__ void load_row(const T* __restrict__ row, bool vec2, T (&x)[B2]) {
  if ((B2 % 2) == 0 && vec2) {
    typedef typename std::conditional<sizeof(T) == 4, float2, double2>::type V2;
    const V2* p = reinterpret_cast<const V2*>(row);
#pragma unroll
    for (int l = 0; l < B2 / 2; ++l) {
      const V2 t = __ldg(p + l);
      x[2 * l] = t.x;
      x[2 * l + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int l = 0; l < B2; ++l) x[l] = __ldg(row + l);
  }
}

// A row of n <= B2 values (scalar loads; the rest of x is zero).
template <typename T, int B2>
__device__ __forceinline__ void load_row_n(const T* __restrict__ row, uint32_t n, T (&x)[B2]) {
#pragma unroll
  for (int l = 0; l < B2; ++l) x[l] = (uint32_t)l < n ? __ldg(row + l) : T(0);
}

__device__ __forceinline__ bool full_block(const Geo& g, uint64_t b, uint64_t c[3]) {
  block_coords(g, b, c[0], c[1], c[2]);
  return (c[0] + 1) * g.B[0] <= g.d[0] && (c[1] + 1) * g.B[1] <= g.d[1] && (c[2] + 1) * g.B[2] <= g.d[2];
}

}  // namespace

// Generic path: edge blocks (or every block when `all`), runtime extents.
template <typename T, int NDIM>
__device__ __forceinline__ void prep_generic(const T* __restrict__ field, const Geo& g, const Ws& w, bool all,
                                             uint64_t count, uint64_t cta, unsigned char* smem) {
  State* st = w.st;
  const uint32_t tid = threadIdx.x;
  const uint64_t e = cta * blockDim.x + tid;
  const bool rel = g.eb_mode == 1;
  T mn = T(1.0 / 0.0), mx = T(-1.0 / 0.0);
  if (e < count) {
    const uint64_t b = all ? e : edge_block(g, e);
    const Box x = block_box(g, b);
    const bool est = g.predictor == 0;
    Walker<float, NDIM> wk;
    wk.base = reinterpret_cast<float*>(smem) + tid;
    wk.stride = blockDim.x;
    wk.B2 = g.B[2];
    wk.sr = g.B[1] * g.B[2];
    const float c0 = 0.5f * (float)(x.e[0] - 1), c1 = 0.5f * (float)(x.e[1] - 1), c2 = 0.5f * (float)(x.e[2] - 1);
    float S0 = 0.0f, Si = 0.0f, Sj = 0.0f, Sl = 0.0f, Elor = 0.0f;
    unsigned long long sum = 0, isum = 0;
    uint32_t k = 0;
    for (uint32_t i = 0; i < x.e[0]; ++i) {
      const float ti = __fsub_rn((float)i, c0);
      for (uint32_t j = 0; j < x.e[1]; ++j) {
        const float tj = __fsub_rn((float)j, c1);
        const T* row = field + row_base(g, x, i, j);
        const bool samp = sample_row(NDIM, i, j, x.e[1]);
        wk.row_start();
        float r0 = 0.0f, rl = 0.0f;
        for (uint32_t l = 0; l < x.e[2]; ++l, ++k) {
          const T v = __ldg(row + l);
          if (rel) minmax<T>(v, mn, mx);
          if (g.abft) cks<T>(v, k, sum, isum);
          const float xr = FT<T>::tofloat(v);
          r0 = __fadd_rn(r0, xr);
          rl = __fadd_rn(rl, __fmul_rn(xr, __fsub_rn((float)l, c2)));
          if (est) {
            wk.load(i, j, l);
            if (samp) {
              const float L = wk.template combine<OpRN<float>>();
              Elor = __fadd_rn(Elor, fabsf(__fsub_rn(xr, L)));
            }
            wk.commit(j, l, xr);
          }
        }
        S0 = __fadd_rn(S0, r0);
        Sl = __fadd_rn(Sl, rl);
        if (NDIM == 3) {
          Si = __fadd_rn(Si, __fmul_rn(r0, ti));
          Sj = __fadd_rn(Sj, __fmul_rn(r0, tj));
        } else if (NDIM == 2) {
          Sj = __fadd_rn(Sj, __fmul_rn(r0, tj));
        }
      }
    }
    float cf[4];
    const float D[3] = {x.e[0] > 1 ? denom(x.P, x.e[0]) : 0.0f, x.e[1] > 1 ? denom(x.P, x.e[1]) : 0.0f,
                        x.e[2] > 1 ? denom(x.P, x.e[2]) : 0.0f};
    const bool finite = coefficients<NDIM>(x.P, x.e, D, S0, Si, Sj, Sl, c0, c1, c2, cf);
    if (g.abft) {
      w.sum_in[b] = sum;
      w.isum_in[b] = isum;
    }
    w.coef[b] = make_float4(cf[0], cf[1], cf[2], cf[3]);
    w.est[b] = make_float2(0.0f, Elor);
    w.pflag[b] = finite ? 1 : 0;
  }
  if (rel) reduce_range<T>(mn, mx, st);
}

template <typename T, int NDIM>
__global__ void __launch_bounds__(128) k_prep(const T* __restrict__ field, Geo g, Ws w, int all, uint64_t count) {
  extern __shared__ __align__(16) unsigned char smem[];
  prep_generic<T, NDIM>(field, g, w, all != 0, count, blockIdx.x, smem);
}

// Batched generic path: the edge blocks (or all blocks) of every job of one dimensionality.
template <typename T, int NDIM>
__global__ void __launch_bounds__(128) k_prep_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Job s_job;
  batch_loop(a, s_job, NoOp(), [&](uint64_t it) {
    prep_generic<T, NDIM>(static_cast<const T*>(s_job.field), s_job.g, s_job.w, !s_job.fast, s_job.gcount, it, smem);
  }, NoOp());
}

// 3D fast blocks whose two planes fit 1 KB per thread are read through shared memory: the
// next plane is copied asynchronously (cp.async, 8-byte units) while the current one is walked,
// so the row loads no longer wait on HBM one after another.
template <typename T, int NDIM, int B1, int B2>
struct PrepStage {
  static constexpr int U = B2 * (int)sizeof(T) / 8;  // 8-byte units per row
  static constexpr bool on = NDIM == 3 && (B2 * sizeof(T)) % 8 == 0 && 2 * B1 * B2 * sizeof(T) <= 1024;
  static constexpr size_t bytes(uint32_t threads) { return on ? (size_t)2 * B1 * U * 8 * threads : 0; }
};

__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}

constexpr int kPrepCta = 128;  // threads of the fast prep kernels' CTAs

// Fast path: full blocks of a compile-time shape B0 x B1 x B2 (leading 1 for 2D). EDGE: the
// edge blocks of such a field (e-th of `count`), walked with the same code at their actual
// extents (at most B0 x B1 x B2; the unrolled row skips what lies outside, and nothing outside
// enters a sum).
template <typename T, int NDIM, int B0, int B1, int B2, bool EDGE = false>
__device__ __forceinline__ void prep_fast(const T* __restrict__ field, const Geo& g, const Ws& w, int vec2,
                                          uint64_t cta, unsigned char* stage, uint64_t count = 0) {
  State* st = w.st;
  const uint32_t tid = threadIdx.x;
  const uint64_t tix = cta * kPrepCta + tid;
  const bool rel = g.eb_mode == 1;
  const bool est = g.predictor == 0;
  T mn = T(1.0 / 0.0), mx = T(-1.0 / 0.0);
  uint64_t c[3];
  uint64_t b = tix;
  bool on;
  Box bx;
  if (EDGE) {
    on = tix < count;
    if (on) {
      b = edge_block(g, tix);
      bx = block_box(g, b);
    }
  } else {
    on = b < g.nb && full_block(g, b, c);
  }
  if (on) {
    const uint32_t n0 = EDGE ? bx.e[0] : B0, n1 = EDGE ? bx.e[1] : B1, n2 = EDGE ? bx.e[2] : B2;
    const uint32_t P = n0 * n1 * n2;
    const T* blk = EDGE ? field + row_base(g, bx, 0, 0) : field + (c[0] * B0 * g.d[1] + c[1] * B1) * g.d[2] + c[2] * B2;
    const uint64_t si = g.d[1] * g.d[2], sj = g.d[2];
    const float c0 = 0.5f * (float)(n0 - 1), c1 = 0.5f * (float)(n1 - 1), c2 = 0.5f * (float)(n2 - 1);
    float S0 = 0.0f, Si = 0.0f, Sj = 0.0f, Sl = 0.0f, Elor = 0.0f;
    unsigned long long sum = 0, isum = 0;
    // E_lor neighbours of the sample rows: the previous row of this plane (brow) and, in 3D,
    // rows (s, s-1) of the previous plane (pa, pb), saved while that plane was walked (na, nb).
    float brow[B2], pa[B2], pb[B2], na[B2], nb[B2];
#pragma unroll
    for (int l = 0; l < B2; ++l) pa[l] = pb[l] = na[l] = nb[l] = 0.0f;
    using ST = PrepStage<T, NDIM, B1, B2>;
    const bool staged = !EDGE && ST::on && vec2;
    // unit u of row r of buffer f of this thread: 8 bytes at ((f*B1 + r)*U + u)*kPrepCta + tid
    unsigned long long* my = reinterpret_cast<unsigned long long*>(stage) + tid;
    auto unit = [&](int f, int r, int u) { return my + ((f * B1 + r) * ST::U + u) * kPrepCta; };
    auto issue_plane = [&](int i) {
#pragma unroll 1
      for (int r = 0; r < B1; ++r)
#pragma unroll
        for (int u = 0; u < ST::U; ++u)
          cp_async8(unit(i & 1, r, u), reinterpret_cast<const unsigned char*>(blk + (uint64_t)i * si + (uint64_t)r * sj) + 8 * u);
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (ST::on && staged) issue_plane(0);
#pragma unroll 1
    for (int i = 0; i < (int)n0; ++i) {
      const float ti = __fsub_rn((float)i, c0);
      const int s_cur = i % (int)n1, s_next = (i + 1) % (int)n1;
      if (ST::on && staged) {
        if (i + 1 < B0) {
          issue_plane(i + 1);
          asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
          asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
      }
#pragma unroll 1
      for (int j = 0; j < (int)n1; ++j) {
        const float tj = __fsub_rn((float)j, c1);
        T x[B2];
        if (EDGE) {
          load_row_n<T, B2>(blk + (uint64_t)i * si + (uint64_t)j * sj, n2, x);
        } else if (ST::on && staged) {
#pragma unroll
          for (int u = 0; u < ST::U; ++u) {
            const unsigned long long v = *unit(i & 1, j, u);
            memcpy(reinterpret_cast<unsigned char*>(x) + 8 * u, &v, 8);
          }
        } else {
          load_row<T, B2>(blk + (uint64_t)i * si + (uint64_t)j * sj, vec2, x);
        }
        const uint32_t k0 = (uint32_t)((i * (int)n1 + j) * (int)n2);
        if (rel && !EDGE) {
          // the row's range with NaN-ignoring min/max (fmin/fmax return the other operand of a
          // NaN); a row holding an infinity, or only NaNs, is filtered point by point instead
          T rmn = x[0], rmx = x[0];
#pragma unroll
          for (int l = 1; l < B2; ++l) {
            rmn = fmin(rmn, x[l]);
            rmx = fmax(rmx, x[l]);
          }
          if (FT<T>::finite(rmn) && FT<T>::finite(rmx)) {
            mn = rmn < mn ? rmn : mn;
            mx = rmx > mx ? rmx : mx;
          } else {
#pragma unroll
            for (int l = 0; l < B2; ++l) minmax<T>(x[l], mn, mx);
          }
        }
        float r0 = 0.0f, rl = 0.0f;
#pragma unroll
        for (int l = 0; l < B2; ++l) {
          if (EDGE && l >= (int)n2) break;
          const T v = x[l];
          if (rel && EDGE) minmax<T>(v, mn, mx);
          if (g.abft) cks<T>(v, k0 + l, sum, isum);
          const float xr = FT<T>::tofloat(v);
          r0 = __fadd_rn(r0, xr);
          rl = __fadd_rn(rl, __fmul_rn(xr, (float)l - c2));
        }
        if (est) {
          const bool samp = NDIM == 3 ? (j == s_cur) : ((j & 3) == 1);
          if (samp) {
            const bool hj = j > 0;
            float cp = 0.0f, ac = 0.0f, bc = 0.0f, abc = 0.0f;
#pragma unroll
            for (int l = 0; l < B2; ++l) {
              if (EDGE && l >= (int)n2) break;
              const float xr = FT<T>::tofloat(x[l]);
              const float bb = hj ? brow[l] : 0.0f;
              float L;
              if (NDIM == 3) {
                const float a = pa[l], ab = hj ? pb[l] : 0.0f;
                float t = __fadd_rn(a, bb);
                t = __fsub_rn(t, ab);
                t = __fsub_rn(t, ac);
                t = __fsub_rn(t, bc);
                t = __fadd_rn(t, abc);
                L = __fadd_rn(t, cp);
                ac = a;
                abc = ab;
              } else {
                L = __fadd_rn(__fsub_rn(bb, bc), cp);
              }
              bc = bb;
              cp = xr;
              Elor = __fadd_rn(Elor, fabsf(__fsub_rn(xr, L)));
            }
          }
          if (NDIM == 3) {
#pragma unroll
            for (int l = 0; l < B2; ++l) {
              const float xr = FT<T>::tofloat(x[l]);
              if (j == s_next) na[l] = xr;
              if (j + 1 == s_next) nb[l] = xr;
            }
          }
#pragma unroll
          for (int l = 0; l < B2; ++l) brow[l] = FT<T>::tofloat(x[l]);
        }
        S0 = __fadd_rn(S0, r0);
        Sl = __fadd_rn(Sl, rl);
        if (NDIM == 3) {
          Si = __fadd_rn(Si, __fmul_rn(r0, ti));
          Sj = __fadd_rn(Sj, __fmul_rn(r0, tj));
        } else {
          Sj = __fadd_rn(Sj, __fmul_rn(r0, tj));
        }
      }
      if (NDIM == 3) {
#pragma unroll
        for (int l = 0; l < B2; ++l) {
          pa[l] = na[l];
          pb[l] = nb[l];
        }
      }
    }
    const uint32_t e[3] = {n0, n1, n2};
    float cf[4];
    constexpr uint32_t Pc = B0 * B1 * B2;
    constexpr float D0 = denom_c(Pc, B0), D1 = denom_c(Pc, B1), D2 = denom_c(Pc, B2);
    float D[3] = {D0, D1, D2};
    if (EDGE)
      for (int a = 0; a < 3; ++a) D[a] = e[a] > 1 ? denom(P, e[a]) : 0.0f;
    const bool finite = coefficients<NDIM>(P, e, D, S0, Si, Sj, Sl, c0, c1, c2, cf);
    if (g.abft) {
      w.sum_in[b] = sum;
      w.isum_in[b] = isum;
    }
    w.coef[b] = make_float4(cf[0], cf[1], cf[2], cf[3]);
    w.est[b] = make_float2(0.0f, Elor);
    w.pflag[b] = finite ? 1 : 0;
  }
  if (rel) reduce_range<T>(mn, mx, st);
}

template <typename T, int NDIM, int B0, int B1, int B2>
__global__ void __launch_bounds__(128) k_prep_fast(const T* __restrict__ field, Geo g, Ws w, int vec2) {
  extern __shared__ __align__(16) unsigned char stage[];
  prep_fast<T, NDIM, B0, B1, B2>(field, g, w, vec2, blockIdx.x, stage);
}

// Edge blocks of a field whose full blocks take k_prep_fast (compact enumeration, one thread
// per edge block).
template <typename T, int NDIM, int B0, int B1, int B2>
__global__ void __launch_bounds__(128) k_prep_edge(const T* __restrict__ field, Geo g, Ws w, uint64_t count) {
  prep_fast<T, NDIM, B0, B1, B2, true>(field, g, w, 0, blockIdx.x, nullptr, count);
}

template <typename T, int NDIM, int B0, int B1, int B2>
__global__ void __launch_bounds__(128) k_prep_fast_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char stage[];
  __shared__ Job s_job;
  batch_loop(a, s_job, NoOp(), [&](uint64_t it) {
    prep_fast<T, NDIM, B0, B1, B2>(static_cast<const T*>(s_job.field), s_job.g, s_job.w, s_job.vec2, it, stage);
  }, NoOp());
}

// The absolute bound: value-range relative (rel * (max - min) over finite values, rounded
// to the dtype; the user's value when the range is empty or zero) or absolute.
template <typename T>
__device__ __forceinline__ void bound_of(const Geo& g, State* st) {
  double ebd = g.e;
  const unsigned long long mi = st->min_key, ma = st->max_key;
  if (g.eb_mode == 1 && ma != 0ull) {
    const T mn = FT<T>::unkey(~mi), mx = FT<T>::unkey(ma);
    if (mx > mn) ebd = __dmul_rn(g.e, __dsub_rn((double)mx, (double)mn));
  }
  T eb;
  if (sizeof(T) == 4) eb = (T)__double2float_rn(ebd);
  else eb = (T)ebd;
  if (!FT<T>::is_normal_pos(eb)) atomicOr(&st->error, ERR_EB);
  st->eb = (double)eb;
  if (g.enc) {
    const CoefSteps cs = coef_steps(g, (double)eb);
    for (int a = 0; a < 4; ++a) {
      st->cstep[a] = cs.step[a];
      st->cinv[a] = cs.inv[a];
    }
  }
}

template <typename T>
__global__ void k_bound(Geo g, State* st) { bound_of<T>(g, st); }

// One thread per job of a batch.
__global__ void k_bound_batch(const Job* jobs, uint32_t n) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const Job& jb = jobs[j];
  if (jb.g.dtype == 0) bound_of<float>(jb.g, jb.w.st);
  else bound_of<double>(jb.g, jb.w.st);
}

// EDGE_ONLY: the edge blocks (on the side stream), else the full blocks.
template <typename T, int NDIM, int B0, int B1, int B2>
static void run_fast(const void* field, const Geo& g, const Ws& w, const Launch& L, bool edge_only) {
  if (edge_only) {
    const uint64_t count = edge_count(g);
    if (!count) return;
    k_prep_edge<T, NDIM, B0, B1, B2><<<(unsigned)((count + 127) / 128), 128, 0, L.stream>>>(
        static_cast<const T*>(field), g, w, count);
    note_launch();
    return;
  }
  const size_t smem = PrepStage<T, NDIM, B1, B2>::bytes(128);
  auto kern = k_prep_fast<T, NDIM, B0, B1, B2>;
  allow_smem(reinterpret_cast<const void*>(kern), smem);
  const bool vec2 = (B2 % 2 == 0) && (g.d[2] % 2 == 0) && (reinterpret_cast<uintptr_t>(field) % (2 * sizeof(T)) == 0);
  kern<<<(unsigned)((g.nb + 127) / 128), 128, smem, L.stream>>>(static_cast<const T*>(field), g, w, vec2 ? 1 : 0);
  note_launch();
}

// The full-block shapes with a fast path (cubes 4..16 in 3D, squares 8/12/16 in 2D).
static bool has_fast(const Geo& g) {
  if (g.ndim == 3 && g.B[0] == g.B[1] && g.B[1] == g.B[2])
    return g.B[2] == 4 || g.B[2] == 6 || g.B[2] == 8 || g.B[2] == 10 || g.B[2] == 12 || g.B[2] == 16;
  if (g.ndim == 2 && g.B[1] == g.B[2]) return g.B[2] == 8 || g.B[2] == 12 || g.B[2] == 16;
  return false;
}

template <typename T>
static bool try_fast(const void* field, const Geo& g, const Ws& w, const Launch& L, bool edge_only) {
  if (g.ndim == 3 && g.B[0] == g.B[1] && g.B[1] == g.B[2]) {
    switch (g.B[2]) {
      case 4: run_fast<T, 3, 4, 4, 4>(field, g, w, L, edge_only); return true;
      case 6: run_fast<T, 3, 6, 6, 6>(field, g, w, L, edge_only); return true;
      case 8: run_fast<T, 3, 8, 8, 8>(field, g, w, L, edge_only); return true;
      case 10: run_fast<T, 3, 10, 10, 10>(field, g, w, L, edge_only); return true;
      case 12: run_fast<T, 3, 12, 12, 12>(field, g, w, L, edge_only); return true;
      case 16: run_fast<T, 3, 16, 16, 16>(field, g, w, L, edge_only); return true;
      default: return false;
    }
  }
  if (g.ndim == 2 && g.B[1] == g.B[2]) {
    switch (g.B[2]) {
      case 8: run_fast<T, 2, 1, 8, 8>(field, g, w, L, edge_only); return true;
      case 12: run_fast<T, 2, 1, 12, 12>(field, g, w, L, edge_only); return true;
      case 16: run_fast<T, 2, 1, 16, 16>(field, g, w, L, edge_only); return true;
      default: return false;
    }
  }
  return false;
}

template <typename T, int NDIM>
static void run_generic(const void* field, const Geo& g, const Ws& w, bool all, const Launch& L) {
  const uint32_t threads = 128;
  const uint64_t count = all ? g.nb : edge_count(g);
  if (!count) return;
  const size_t smem = (g.predictor == 0) ? (size_t)walker_slots(g.ndim, g.B) * threads * sizeof(float) : 0;
  allow_smem(reinterpret_cast<const void*>(k_prep<T, NDIM>), smem);
  k_prep<T, NDIM><<<(unsigned)((count + threads - 1) / threads), threads, smem, L.stream>>>(
      static_cast<const T*>(field), g, w, all ? 1 : 0, count);
  note_launch();
}

template <typename T>
static void launch_prep_t(const void* field, const Geo& g, const Ws& w, const Launch& L) {
  if (g.nb) {
    // edge blocks on the side stream, concurrently with the full blocks
    Fork fk(L);
    const Launch Ls = fk.side_launch(L);
    const bool fast = has_fast(g);
    if (fast) {
      try_fast<T>(field, g, w, Ls, true);  // edge blocks: the same walk at their extents
      try_fast<T>(field, g, w, L, false);
    } else if (g.ndim == 3) {
      run_generic<T, 3>(field, g, w, true, L);
    } else if (g.ndim == 2) {
      run_generic<T, 2>(field, g, w, true, L);
    } else {
      run_generic<T, 1>(field, g, w, true, L);
    }
    fk.join();
  }
  k_bound<T><<<1, 1, 0, L.stream>>>(g, w.st);
  note_launch();
}

// ---------------------------------------------------------------- batched launches
template <class K>
static unsigned batch_grid(K kern, uint32_t threads, size_t smem, uint64_t items, const Launch& L) {
  const int occ = occupancy(reinterpret_cast<const void*>(kern), (int)threads, smem);
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(items, (uint64_t)occ * L.sms));
}

template <typename T, int NDIM, int B0, int B1, int B2>
static void batch_fast_t(const BatchArgs& a, const Launch& L) {
  auto kern = k_prep_fast_batch<T, NDIM, B0, B1, B2>;
  const size_t smem = PrepStage<T, NDIM, B1, B2>::bytes(128);
  const unsigned grid = batch_grid(kern, 128, smem, a.start[a.n], L);
  kern<<<grid, 128, smem, L.stream>>>(a);
  note_launch();
}

template <typename T>
static bool batch_fast_dt(int ndim, uint32_t B, const BatchArgs& a, const Launch& L) {
  if (ndim == 3) {
    switch (B) {
      case 4: batch_fast_t<T, 3, 4, 4, 4>(a, L); return true;
      case 6: batch_fast_t<T, 3, 6, 6, 6>(a, L); return true;
      case 8: batch_fast_t<T, 3, 8, 8, 8>(a, L); return true;
      case 10: batch_fast_t<T, 3, 10, 10, 10>(a, L); return true;
      case 12: batch_fast_t<T, 3, 12, 12, 12>(a, L); return true;
      case 16: batch_fast_t<T, 3, 16, 16, 16>(a, L); return true;
      default: return false;
    }
  }
  if (ndim == 2) {
    switch (B) {
      case 8: batch_fast_t<T, 2, 1, 8, 8>(a, L); return true;
      case 12: batch_fast_t<T, 2, 1, 12, 12>(a, L); return true;
      case 16: batch_fast_t<T, 2, 1, 16, 16>(a, L); return true;
      default: return false;
    }
  }
  return false;
}

bool batch_prep_fast(int dtype, int ndim, uint32_t B, const BatchArgs& a, const Launch& L) {
  return dtype == 0 ? batch_fast_dt<float>(ndim, B, a, L) : batch_fast_dt<double>(ndim, B, a, L);
}

template <typename T, int NDIM>
static void batch_generic_t(const BatchArgs& a, size_t smem, const Launch& L) {
  auto kern = k_prep_batch<T, NDIM>;
  const unsigned grid = batch_grid(kern, 128, smem, a.start[a.n], L);
  kern<<<grid, 128, smem, L.stream>>>(a);
  note_launch();
}

void batch_prep_generic(int dtype, int ndim, const BatchArgs& a, size_t smem, const Launch& L) {
  if (dtype == 0) {
    if (ndim == 3) batch_generic_t<float, 3>(a, smem, L);
    else if (ndim == 2) batch_generic_t<float, 2>(a, smem, L);
    else batch_generic_t<float, 1>(a, smem, L);
  } else {
    if (ndim == 3) batch_generic_t<double, 3>(a, smem, L);
    else if (ndim == 2) batch_generic_t<double, 2>(a, smem, L);
    else batch_generic_t<double, 1>(a, smem, L);
  }
}

void batch_bound(const Job* jobs, uint32_t n, const Launch& L) {
  k_bound_batch<<<(n + 63) / 64, 64, 0, L.stream>>>(jobs, n);
  note_launch();
}

bool prep_has_fast(const Geo& g) { return has_fast(g); }

void launch_bound(const Geo& g, State* st, const Launch& L) {
  if (g.dtype == 0) k_bound<float><<<1, 1, 0, L.stream>>>(g, st);
  else k_bound<double><<<1, 1, 0, L.stream>>>(g, st);
  note_launch();
}

void launch_prep(const void* field, const Geo& g, const Ws& w, const Launch& L) {
  if (g.dtype == 0) launch_prep_t<float>(field, g, w, L);
  else launch_prep_t<double>(field, g, w, L);
}

}  // namespace sdcsz
