// K1: prediction preparation and input checksums (Alg. 1 lines 1-7 of the paper).
//
// One thread per block, a warp per 32 consecutive blocks. A single pass over the block
// computes, from the input as it is when compression starts:
//   * sum_in / isum_in over the block's 32-bit words (Alg. 1 lines 3-4; Sec. 3.2, 5.4),
//   * the regression sums and the closed-form least-squares coefficients (line 2),
//   * the Lorenzo estimate E_lor on the original values (lines 6-7),
//   * the value range for the value-range relative bound;
// a second pass over the same block (L1/L2 resident) adds the regression estimate E_reg.
// The last CTA to finish turns the global range into the absolute bound eb.
#include "sdcsz_internal.cuh"

namespace sdcsz {

template <typename T, int NDIM>
__global__ void __launch_bounds__(128) k_prep(const T* __restrict__ field, Geo g, Ws w) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_min[4], s_max[4];
  State* st = w.st;
  const uint32_t tid = threadIdx.x;
  const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + tid;
  const bool rel = g.eb_mode == 1;
  unsigned long long kmin_inv = 0ull, kmax = 0ull;  // 0 = no finite value seen

  if (b < g.nb) {
    const Box x = block_box(g, b);
    const bool est = g.predictor == 0;
    Walker<float, NDIM> wk;
    wk.base = reinterpret_cast<float*>(smem) + tid;
    wk.stride = blockDim.x;
    wk.B2 = g.B[2];
    wk.sr = g.B[1] * g.B[2];
    // centre of each active axis (half-integers, exact in fp32)
    const float c0 = 0.5f * (float)(x.e[0] - 1), c1 = 0.5f * (float)(x.e[1] - 1), c2 = 0.5f * (float)(x.e[2] - 1);
    float S0 = 0.0f, Si = 0.0f, Sj = 0.0f, Sl = 0.0f, Elor = 0.0f;
    unsigned long long sum = 0, isum = 0;
    uint32_t k = 0;
    for (uint32_t i = 0; i < x.e[0]; ++i) {
      const float ti = __fsub_rn((float)i, c0);
      for (uint32_t j = 0; j < x.e[1]; ++j) {
        const float tj = __fsub_rn((float)j, c1);
        const T* row = field + row_base(g, x, i, j);
        wk.row_start();
        for (uint32_t l = 0; l < x.e[2]; ++l, ++k) {
          const T v = __ldg(row + l);
          if (rel && FT<T>::finite(v)) {
            const unsigned long long key = FT<T>::key(v);
            kmin_inv = max(kmin_inv, ~key);
            kmax = max(kmax, key);
          }
          if (g.abft) add_words<T>(v, k, sum, isum);
          const float xr = FT<T>::tofloat(v);
          const float tl = __fsub_rn((float)l, c2);
          S0 = __fadd_rn(S0, xr);
          if (NDIM == 3) {
            Si = __fadd_rn(Si, __fmul_rn(xr, ti));
            Sj = __fadd_rn(Sj, __fmul_rn(xr, tj));
            Sl = __fadd_rn(Sl, __fmul_rn(xr, tl));
          } else if (NDIM == 2) {
            Sj = __fadd_rn(Sj, __fmul_rn(xr, tj));
            Sl = __fadd_rn(Sl, __fmul_rn(xr, tl));
          } else {
            Sl = __fadd_rn(Sl, __fmul_rn(xr, tl));
          }
          if (est) {
            wk.load(i, j, l);
            const float L = wk.template combine<OpRN<float>>();
            Elor = __fadd_rn(Elor, fabsf(__fsub_rn(xr, L)));
            wk.commit(j, l, xr);
          }
        }
      }
    }
    // closed-form least squares on the block grid: slope = sum x*(c - ctr) / sum (c - ctr)^2
    const float Pf = (float)x.P;
    auto denom = [&](uint32_t ed) -> float {
      return __double2float_rn(__ddiv_rn(__dmul_rn((double)x.P, __dsub_rn(__dmul_rn((double)ed, (double)ed), 1.0)), 12.0));
    };
    float cf[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const float mean = __fdiv_rn(S0, Pf);
    if (NDIM == 3) {
      cf[0] = x.e[0] > 1 ? __fdiv_rn(Si, denom(x.e[0])) : 0.0f;
      cf[1] = x.e[1] > 1 ? __fdiv_rn(Sj, denom(x.e[1])) : 0.0f;
      cf[2] = x.e[2] > 1 ? __fdiv_rn(Sl, denom(x.e[2])) : 0.0f;
      float acc = __fmul_rn(cf[0], c0);
      acc = __fadd_rn(acc, __fmul_rn(cf[1], c1));
      acc = __fadd_rn(acc, __fmul_rn(cf[2], c2));
      cf[3] = __fsub_rn(mean, acc);
    } else if (NDIM == 2) {
      cf[0] = x.e[1] > 1 ? __fdiv_rn(Sj, denom(x.e[1])) : 0.0f;
      cf[1] = x.e[2] > 1 ? __fdiv_rn(Sl, denom(x.e[2])) : 0.0f;
      float acc = __fmul_rn(cf[0], c1);
      acc = __fadd_rn(acc, __fmul_rn(cf[1], c2));
      cf[2] = __fsub_rn(mean, acc);
    } else {
      cf[0] = x.e[2] > 1 ? __fdiv_rn(Sl, denom(x.e[2])) : 0.0f;
      cf[1] = __fsub_rn(mean, __fmul_rn(cf[0], c2));
    }
    bool finite = true;
    for (int a = 0; a <= NDIM; ++a) finite = finite && isfinite(cf[a]);
    float Ereg = 0.0f;
    if (est && finite) {
      for (uint32_t i = 0; i < x.e[0]; ++i)
        for (uint32_t j = 0; j < x.e[1]; ++j) {
          const T* row = field + row_base(g, x, i, j);
          for (uint32_t l = 0; l < x.e[2]; ++l) {
            const float xr = FT<T>::tofloat(__ldg(row + l));
            const float f = regress<float, NDIM, OpRN<float>>(cf, i, j, l);
            Ereg = __fadd_rn(Ereg, fabsf(__fsub_rn(xr, f)));
          }
        }
    }
    if (g.abft) {
      w.sum_in[b] = sum;
      w.isum_in[b] = isum;
    }
    w.coef[b] = make_float4(cf[0], cf[1], cf[2], cf[3]);
    w.est[b] = make_float2(Ereg, Elor);
    w.pflag[b] = finite ? 1 : 0;
  }

  // value range: warp, CTA, then grid (atomics on monotone keys)
  if (rel) {
    for (int o = 16; o > 0; o >>= 1) {
      kmin_inv = max(kmin_inv, __shfl_xor_sync(0xffffffffu, kmin_inv, o));
      kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    if ((tid & 31) == 0) {
      s_min[tid >> 5] = kmin_inv;
      s_max[tid >> 5] = kmax;
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (rel) {
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
    __threadfence();
    const unsigned int done = atomicAdd(&st->k1_done, 1u);
    if (done == gridDim.x - 1) {
      // last CTA: the absolute bound (value-range relative, or the user's absolute bound)
      __threadfence();
      double ebd = g.e;
      const unsigned long long mi = atomicAdd(&st->min_key, 0ull), ma = atomicAdd(&st->max_key, 0ull);
      if (rel && ma != 0ull) {
        const T mn = FT<T>::unkey(~mi), mx = FT<T>::unkey(ma);
        if (mx > mn) ebd = __dmul_rn(g.e, __dsub_rn((double)mx, (double)mn));
      }
      T eb;
      if (sizeof(T) == 4) eb = (T)__double2float_rn(ebd);
      else eb = (T)ebd;
      if (!FT<T>::is_normal_pos(eb)) atomicOr(&st->error, ERR_EB);
      st->eb = (double)eb;
    }
  }
}

template <typename T, int NDIM>
static void run_prep(const void* field, const Geo& g, const Ws& w, const Launch& L) {
  const uint32_t threads = 128;
  const uint64_t grid = g.nb ? (g.nb + threads - 1) / threads : 1;
  const size_t smem = (g.predictor == 0) ? (size_t)walker_slots(g.ndim, g.B) * threads * sizeof(float) : 0;
  cudaFuncSetAttribute(k_prep<T, NDIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_prep<T, NDIM><<<(unsigned)grid, threads, smem, L.stream>>>(static_cast<const T*>(field), g, w);
}

void launch_prep(const void* field, const Geo& g, const Ws& w, const Launch& L) {
  if (g.dtype == 0) {
    if (g.ndim == 3) run_prep<float, 3>(field, g, w, L);
    else if (g.ndim == 2) run_prep<float, 2>(field, g, w, L);
    else run_prep<float, 1>(field, g, w, L);
  } else {
    if (g.ndim == 3) run_prep<double, 3>(field, g, w, L);
    else if (g.ndim == 2) run_prep<double, 2>(field, g, w, L);
    else run_prep<double, 1>(field, g, w, L);
  }
}

}  // namespace sdcsz
