// K2: prediction, quantization and block checksums (the predictor choice and the per-block
// prediction loop of Algorithm 1 of the paper).
//
// One thread per block, a warp per 32 consecutive blocks, persistent CTAs. Per block:
//   * predictor choice from the K1 estimates (indicator[i]),
//   * one pass over the block in its sequential order: prediction evaluated twice
//     (f_dup), linear-scaling quantization with the bin-range check, reconstruction evaluated
//     twice (dec_dup), the machine-epsilon double check (Sec. 4.1.2), the code, sum_q/isum_q
//     and sum_dc, and the input words' checksums;
//   * Algorithm 1's input check before prediction is done speculatively: the words used by the pass are
//     summed on the fly and compared with sum_in/isum_in at the end; a mismatch (a memory
//     error since K1) is located, repaired, and the block is run again with the repaired
//     value, so the output equals that of an error-free run.
// Two kernels: a fast path for full blocks of the common shapes (compile-time block edges,
// the fastest-axis row unrolled in registers, the Lorenzo neighbours of the previous row in
// registers and of the previous plane in one in-place shared-memory plane per thread), and a
// generic path for edge blocks and other shapes. Codes and unpredictable values go to
// warp-interleaved staging arrays (coalesced stores); the code histogram is privatised in
// shared memory around the central bin.
#pragma once

#include <algorithm>
#include <type_traits>

#include "sdcsz_internal.cuh"

namespace sdcsz {
namespace kpred {
namespace {

constexpr uint32_t kNone = 0xffffffffu;

struct PassRes {
  unsigned long long sw, isw;  // checksums of the input words used
  unsigned long long isq, sdc; // isum_q, sum_dc
  uint32_t sq, nun, dup;       // sum_q (< 2^28), unpredictables, duplicate mismatches (voting walk)
  uint32_t mm;                 // OR of (primary ^ duplicate) bits over the block (unvoted walk)
};

struct Hist {
  uint32_t* s;            // shared window
  unsigned long long* g;  // global histogram
  uint32_t lo, hi;
  __device__ __forceinline__ void add(uint32_t code, uint32_t cnt) const {
    if (code - lo < hi - lo) atomicAdd(&s[code - lo], cnt);
    else atomicAdd(&g[code], (unsigned long long)cnt);
  }
  __device__ __forceinline__ void sub1(uint32_t code) const {
    if (code - lo < hi - lo) atomicSub(&s[code - lo], 1u);
    else atomicAdd(&g[code], ~0ull);
  }
};

// Histogram front end: the central bin (prediction within one bin) is counted in a register
// without branching; every other code costs one shared (or global) atomic.
struct Run {
  uint32_t centre, n = 0;
  __device__ __forceinline__ explicit Run(uint32_t R) : centre(R) {}
  __device__ __forceinline__ void push(uint32_t c, const Hist& h) {
    n += (c == centre);
    if (c != centre) h.add(c, 1u);
  }
  __device__ __forceinline__ void flush(const Hist& h) {
    if (n) h.add(centre, n);
    n = 0;
  }
};

// acc += a * b with one 32x32 -> 64 multiply-add
__device__ __forceinline__ void mad_wide(unsigned long long& acc, uint32_t a, uint32_t b) {
  asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

template <typename T>
__device__ __forceinline__ void cks_words(T v, uint32_t k, unsigned long long& sum, unsigned long long& isum) {
  const uint32_t w0 = FT<T>::lo(v);
  if (FT<T>::W == 1) {
    mad_wide(sum, w0, 1u);
    mad_wide(isum, w0, k + 1);
  } else {
    const uint32_t w1 = FT<T>::hi(v);
    mad_wide(sum, w0, 1u);
    mad_wide(sum, w1, 1u);
    mad_wide(isum, w0, 2 * k + 1);
    mad_wide(isum, w1, 2 * k + 2);
  }
}

template <typename T>
__device__ __forceinline__ void sum_words(T v, unsigned long long& sum) {
  mad_wide(sum, FT<T>::lo(v), 1u);
  if (FT<T>::W == 2) mad_wide(sum, FT<T>::hi(v), 1u);
}

// Algorithm 1 for one point with its (already duplicated) prediction: linear-scaling
// quantization, reconstruction with dec_dup, and the machine-epsilon double check.
// Returns the code (0 = unpredictable) and the value later points are predicted from.
// An unpredictable point decompresses to its value, truncated to the mantissa bits the bound
// needs in the compact encoding (texp = floor(log2 eb)); texp = kNoTrunc keeps it whole.
//
// Two forms of the duplicate checks (f_dup, dec_dup). VOTE (the walk that soft-error records
// reach, and every re-run): a disagreement is settled at once by a third evaluation and
// counted. Otherwise the walk only ORs the XOR of the two results into `mm`, without a branch;
// the caller runs a block whose mask is not zero again with VOTE, which settles the
// disagreement the same way. Both results come from the same operations on the same operands,
// so without a fault they agree bit for bit, in range or not.
template <typename T, bool ABFT, bool VOTE, bool CMP>
__device__ __forceinline__ uint32_t quantize(T v, T pred, T eb, T inv2, T Rh, uint32_t R, bool hit_r, uint32_t bitr,
                                             T& xr, uint32_t& dup, uint32_t& mm, int texp) {
  const T diff = FT<T>::sub(v, pred);
  const T t = FT<T>::mul(FT<T>::absv(diff), inv2);
  const bool inr = t < Rh;
  const int m = FT<T>::trunc_i(FT<T>::add(t, T(0.5)));
  const int q = (diff < T(0)) ? -m : m;
  const T tq = FT<T>::fromi(2 * q);
  T xd = FT<T>::add(pred, FT<T>::mul(tq, eb));
  if (ABFT) {
    if (VOTE && hit_r) xd = FT<T>::flip(xd, bitr);
    const T x2 = FT<T>::add_v(pred, FT<T>::mul_v(tq, eb));
    if (VOTE) {
      if (inr && !FT<T>::same(xd, x2)) {
        xd = FT<T>::add_v(pred, FT<T>::mul_v(tq, eb));
        ++dup;
      }
    } else {
      mm |= FT<T>::diffbits(xd, x2);
    }
  }
  const bool ok = inr && (FT<T>::absv(FT<T>::sub(v, xd)) <= eb);
  if (ok) xr = xd;
  else xr = CMP ? truncated<T>(v, texp) : v;
  return ok ? (uint32_t)(q + (int)R) : 0u;
}

// f_dup for a prediction computed by `prim` (rounded intrinsics) and `dupf` (volatile PTX);
// VOTE as for quantize.
template <typename T, bool ABFT, bool VOTE, class F1, class F2>
__device__ __forceinline__ T dup_pred(F1 prim, F2 dupf, bool hit_p, uint32_t bitp, uint32_t& dup, uint32_t& mm) {
  T pred = prim();
  if (ABFT) {
    if (VOTE && hit_p) pred = FT<T>::flip(pred, bitp);
    const T p2 = dupf();
    if (VOTE) {
      if (!FT<T>::same(pred, p2)) {
        pred = dupf();
        ++dup;
      }
    } else {
      mm |= FT<T>::diffbits(pred, p2);
    }
  }
  return pred;
}

struct Hooks {
  uint32_t kp, bitp, kr, bitr, kfix;
  bool rewalk;  // test record: take the re-walk of a disagreeing block without a disagreement
  int texp;  // truncation exponent of unpredictable values (kNoTrunc: raw encoding)
};

// ---------------------------------------------------------------- generic path
template <typename T, int NDIM, bool REG, bool ABFT>
__device__ __noinline__ PassRes generic_pass(const T* __restrict__ field, const Geo& g, const Box& x, uint64_t b,
                                             const T* cT, Walker<T, NDIM>& wk, T eb, T inv2, T Rh,
                                             uint16_t* __restrict__ codes, T* __restrict__ ustage, const Hist& h,
                                             const Hooks hk, T xfix) {
  PassRes r = {0, 0, 0, 0, 0, 0, 0, 0};
  Run run(g.R);
  uint64_t ci = code_index(b, g.P, 0);  // unpredictable staging (one slot per point)
  uint32_t k = 0;
  for (uint32_t i = 0; i < x.e[0]; ++i) {
    for (uint32_t j = 0; j < x.e[1]; ++j) {
      const T* row = field + row_base(g, x, i, j);
      if (!REG) wk.row_start();
      for (uint32_t l = 0; l < x.e[2]; ++l, ++k, ci += 32) {
        const T v = (k == hk.kfix) ? xfix : __ldg(row + l);
        if (ABFT) cks_words<T>(v, k, r.sw, r.isw);
        if (!REG) wk.load(i, j, l);
        const T pred = dup_pred<T, ABFT, true>(
            [&] { return REG ? regress<T, NDIM, OpRN<T>>(cT, i, j, l) : wk.template combine<OpRN<T>>(); },
            [&] { return REG ? regress<T, NDIM, OpV<T>>(cT, i, j, l) : wk.template combine<OpV<T>>(); },
            k == hk.kp, hk.bitp, r.dup, r.mm);
        T xr;
        const uint32_t code = quantize<T, ABFT, true, true>(v, pred, eb, inv2, Rh, g.R, k == hk.kr, hk.bitr, xr, r.dup,
                                                      r.mm, hk.texp);
        codes[code_pos(b, g.P, k)] = (uint16_t)code;
        if (!code) {
          ustage[ci] = v;
          ++r.nun;
        }
        if (ABFT) {
          r.sq += code;
          mad_wide(r.isq, code, k + 1);
          sum_words<T>(xr, r.sdc);
        }
        run.push(code, h);
        if (!REG) wk.commit(j, l, xr);
      }
    }
  }
  run.flush(h);
  return r;
}

// ---------------------------------------------------------------- fast path (full blocks)
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

// The 3D (2D) Lorenzo prediction from its seven (three) neighbours, in the reading's order:
// the previous point of the row (c) last.
template <typename T, int NDIM, class Op>
__device__ __forceinline__ T lorenzo_of(T a, T bb, T ab, T ac, T bc, T abc, T c) {
  if (NDIM == 3) {
    T s = Op::add(a, bb);
    s = Op::sub(s, ab);
    s = Op::sub(s, ac);
    s = Op::sub(s, bc);
    s = Op::add(s, abc);
    return Op::add(s, c);
  }
  if (NDIM == 2) return Op::add(Op::sub(a, ac), c);
  return c;
}

// One full block with compile-time edges. `blk` points at the block origin in the field,
// `plane` at this thread's shared-memory slot 0 (3D Lorenzo only; slot stride kCta).
// HOOK: the voting walk that also applies the soft-error records in `hk` (VOTE of quantize);
// otherwise duplicate disagreements only collect in the result's mask.
// EDGE: a block cut by the field boundary, extents e0 x e1 x e2 at most B0 x B1 x B2 (the
// loops keep their compile-time bounds and skip what lies outside; codes are paired by the
// block-local index, which need not start a row on a pair).
//
// Central rows (the unvoted walk of full blocks): a row is first walked on the assumption that
// every point lands in the central bin, where quantize() gives code R and x' = pred + 0
// exactly (see central_threshold). The assumption holds for a point when |x - pred| <= D*;
// if it holds for every point of the row in every lane of the warp, the row's codes, x' and
// checksums are the ones quantize() would give (the codes all R, sum_q and isum_q in closed
// form) and the row is done; otherwise the row is walked again point by point with the full
// quantizer. Both give the same values bit for bit; only the work differs.
template <typename T, int NDIM, int B0, int B1, int B2, int kCta, bool REG, bool ABFT, bool HOOK, bool CMP,
          bool EDGE = false>
__device__ __forceinline__ PassRes fast_pass(const T* __restrict__ blk, uint64_t si, uint64_t sj, bool vec2,
                                             const T* cT, T* plane, T eb, T inv2, T Rh, T dstar, uint32_t R,
                                             uint32_t* __restrict__ pptr, T* __restrict__ uptr, const Hist& h,
                                             const Hooks hk, T xfix, uint32_t e0 = B0, uint32_t e1 = B1,
                                             uint32_t e2 = B2) {
  constexpr bool SPEC = !HOOK && !EDGE;
  PassRes r = {0, 0, 0, 0, 0, 0, 0, 0};
  Run run(R);
  const int n0 = EDGE ? (int)e0 : B0, n1 = EDGE ? (int)e1 : B1;
  uint32_t lowe = 0;  // EDGE: pending low half of a code pair
  if (!REG && NDIM == 3) {
#pragma unroll
    for (int s = 0; s < B1 * B2; ++s) plane[s * kCta] = T(0);
  }
  // regression along the row: the block's products c_l * l, primary and duplicate (the voting
  // walk recomputes them point by point, so a disagreement is settled by a fresh evaluation)
  constexpr int LC = NDIM == 3 ? 2 : (NDIM == 2 ? 1 : 0);
  T clp[B2], clv[B2];
  if (REG && !HOOK) {
#pragma unroll
    for (int l = 0; l < B2; ++l) {
      clp[l] = FT<T>::mul(cT[LC], (T)l);
      clv[l] = FT<T>::mul_v(cT[LC], (T)l);
    }
  }
  const uint32_t RR = R | (R << 16);
  T brow[B2], arow[B2];  // Lorenzo: d[i][j-1][l] and d[i-1][j-1][l] (3D); d[j-1][l] (2D)
#pragma unroll 1
  for (int i = 0; i < n0; ++i) {
#pragma unroll
    for (int l = 0; l < B2; ++l) {
      brow[l] = T(0);
      arow[l] = T(0);
    }
    if (!EDGE && i + 1 < n0) {  // the next plane's rows on their way to L2 while this one is walked
#pragma unroll
      for (int r = 0; r < B1; ++r) prefetch_l2(blk + (uint64_t)(i + 1) * si + (uint64_t)r * sj);
    }
    T xn[B2];
    if (EDGE) load_row_n<T, B2>(blk + (uint64_t)i * si, e2, xn);
    else load_row<T, B2>(blk + (uint64_t)i * si, vec2, xn);
#pragma unroll 1
    for (int j = 0; j < n1; ++j) {
      T x[B2];
#pragma unroll
      for (int l = 0; l < B2; ++l) x[l] = xn[l];
      if (j + 1 < n1) {  // next row
        if (EDGE) load_row_n<T, B2>(blk + (uint64_t)i * si + (uint64_t)(j + 1) * sj, e2, xn);
        else load_row<T, B2>(blk + (uint64_t)i * si + (uint64_t)(j + 1) * sj, vec2, xn);
      }
      const uint32_t k0 = EDGE ? (uint32_t)((i * n1 + j) * (int)e2) : (uint32_t)((i * B1 + j) * B2);
      uint32_t* prow = pptr + (uint64_t)(k0 >> 1) * 32;  // B2 is even: rows start on a pair
      T* urow = uptr + (uint64_t)k0 * 32;
      // the input words' checksums (Algorithm 1's check of the input, verified at the block end)
#pragma unroll
      for (int l = 0; l < B2; ++l) {
        if (EDGE && l >= (int)e2) break;
        if (HOOK && k0 + l == hk.kfix) x[l] = xfix;
        if (ABFT) cks_words<T>(x[l], k0 + l, r.sw, r.isw);
      }
      // regression: (b0*i + b1*j) of this row, twice (primary and duplicate)
      T ra = T(0), rv = T(0);
      if (REG) {
        if (NDIM == 3) {
          ra = FT<T>::add(FT<T>::mul(cT[0], (T)i), FT<T>::mul(cT[1], (T)j));
          rv = FT<T>::add_v(FT<T>::mul_v(cT[0], (T)i), FT<T>::mul_v(cT[1], (T)j));
        } else if (NDIM == 2) {
          ra = FT<T>::mul(cT[0], (T)j);
          rv = FT<T>::mul_v(cT[0], (T)j);
        }
      }
      T* plrow = plane + (uint64_t)j * B2 * kCta;
      bool done = false;
      if (SPEC) {
        T xs[B2], as[B2];
        bool ok = true;
        T c = T(0), ac = T(0), bc = T(0), abc = T(0);
#pragma unroll
        for (int l = 0; l < B2; ++l) {
          T a = T(0), bb = T(0), ab = T(0);
          if (!REG) {
            if (NDIM == 3) {
              a = plrow[l * kCta];
              bb = brow[l];
              ab = arow[l];
            } else if (NDIM == 2) {
              a = brow[l];
            }
          }
          T pred;
          if (REG) pred = NDIM == 1 ? FT<T>::add(clp[l], cT[1]) : FT<T>::add(FT<T>::add(ra, clp[l]), cT[LC + 1]);
          else pred = lorenzo_of<T, NDIM, OpRN<T>>(a, bb, ab, ac, bc, abc, c);
          if (ABFT) {
            T pv;
            if (REG) pv = NDIM == 1 ? FT<T>::add_v(clv[l], cT[1]) : FT<T>::add_v(FT<T>::add_v(rv, clv[l]), cT[LC + 1]);
            else pv = lorenzo_of<T, NDIM, OpV<T>>(a, bb, ab, ac, bc, abc, c);
            r.mm |= FT<T>::diffbits(pred, pv);
          }
          ok = ok && (FT<T>::absv(FT<T>::sub(x[l], pred)) <= dstar);
          const T xr = FT<T>::add(pred, T(0));
          if (ABFT) r.mm |= FT<T>::diffbits(xr, FT<T>::add_v(pred, T(0)));
          xs[l] = xr;
          as[l] = a;
          if (!REG) {
            ac = a;
            bc = bb;
            abc = ab;
            c = xr;
          }
        }
        done = __all_sync(__activemask(), ok);
        if (done) {
#pragma unroll
          for (int l = 0; l < B2; ++l) {
            if (ABFT) sum_words<T>(xs[l], r.sdc);
            if (l & 1) prow[(l >> 1) * 32] = RR;
            if (!REG) {
              if (NDIM == 3) {
                plrow[l * kCta] = xs[l];
                arow[l] = as[l];
                brow[l] = xs[l];
              } else if (NDIM == 2) {
                brow[l] = xs[l];
              }
            }
          }
          if (ABFT) {
            r.sq += (uint32_t)B2 * R;
            r.isq += (unsigned long long)R * ((unsigned long long)B2 * (k0 + 1) + (uint32_t)(B2 * (B2 - 1) / 2));
          }
          run.n += B2;
        }
      }
      if (!done) {
        uint32_t lowc = 0;
        T c = T(0), ac = T(0), bc = T(0), abc = T(0);
#pragma unroll
        for (int l = 0; l < B2; ++l) {
          if (EDGE && l >= (int)e2) break;
          const uint32_t k = k0 + l;
          const T v = x[l];
          T a = T(0), bb = T(0), ab = T(0);
          if (!REG) {
            if (NDIM == 3) {
              a = plrow[l * kCta];
              bb = brow[l];
              ab = arow[l];
            } else if (NDIM == 2) {
              a = brow[l];
            }
          }
          const T L = (T)l;
          const T pred = dup_pred<T, ABFT, HOOK>(
              [&] {
                if (REG) {
                  const T cl = HOOK ? FT<T>::mul(cT[LC], L) : clp[l];
                  if (NDIM == 1) return FT<T>::add(cl, cT[1]);
                  return FT<T>::add(FT<T>::add(ra, cl), cT[LC + 1]);
                }
                return lorenzo_of<T, NDIM, OpRN<T>>(a, bb, ab, ac, bc, abc, c);
              },
              [&] {
                if (REG) {
                  const T cl = HOOK ? FT<T>::mul_v(cT[LC], L) : clv[l];
                  if (NDIM == 1) return FT<T>::add_v(cl, cT[1]);
                  return FT<T>::add_v(FT<T>::add_v(rv, cl), cT[LC + 1]);
                }
                return lorenzo_of<T, NDIM, OpV<T>>(a, bb, ab, ac, bc, abc, c);
              },
              HOOK && k == hk.kp, hk.bitp, r.dup, r.mm);
          T xr;
          const uint32_t code = quantize<T, ABFT, HOOK, CMP>(v, pred, eb, inv2, Rh, R, HOOK && k == hk.kr, hk.bitr, xr,
                                                             r.dup, r.mm, hk.texp);
          if (EDGE) {
            if (k & 1) pptr[(uint64_t)(k >> 1) * 32] = lowe | (code << 16);
            else lowe = code;
          } else {
            if (l & 1) prow[(l >> 1) * 32] = lowc | (code << 16);
            else lowc = code;
          }
          if (!code) urow[l * 32] = v;
          r.nun += (code == 0u);
          if (ABFT) {
            r.sq += code;
            mad_wide(r.isq, code, k + 1);
            sum_words<T>(xr, r.sdc);
          }
          run.push(code, h);
          if (!REG) {
            if (NDIM == 3) {
              plrow[l * kCta] = xr;
              arow[l] = a;
              ac = a;
              bc = bb;
              abc = ab;
              brow[l] = xr;
            } else if (NDIM == 2) {
              ac = a;
              brow[l] = xr;
            }
            c = xr;
          }
        }
      }
    }
  }
  if (EDGE && ((e0 * e1 * e2) & 1)) pptr[(uint64_t)((e0 * e1 * e2) >> 1) * 32] = lowe;  // odd count: last half
  run.flush(h);
  return r;
}

// ---------------------------------------------------------------- kernels
struct Prologue {
  float noise;
  bool reg;
};

// indicator[i]: regression when its estimated error is the smaller one. E_lor comes from K1; E_reg
// (which needs the coefficients) is summed here by `ereg()` just before the block is
// predicted, so its re-read of the block hits the cache.
template <class F>
__device__ __forceinline__ bool choose_reg(const Geo& g, const Ws& w, uint64_t b, bool usable, uint32_t S, float noise,
                                           F ereg) {
  if (!usable) return false;
  if (g.predictor == 2) return true;
  if (g.predictor == 1) return false;
  const float Elor = w.est[b].y;
  const float Ereg = ereg();
  return Ereg < __fadd_rn(Elor, __fmul_rn((float)S, noise));
}

// E_reg = sum |x - f(p)| over the sample rows in local order (fp32; any extents).
// (kfix, xfix): a repaired input value used in place of the stored one.
template <typename T, int NDIM>
__device__ __noinline__ float ereg_generic(const T* __restrict__ field, const Geo& g, const Box& x, float4 c4,
                                           uint32_t kfix, T xfix) {
  const float cf[4] = {c4.x, c4.y, c4.z, c4.w};
  float E = 0.0f;
  uint32_t k = 0;
  for (uint32_t i = 0; i < x.e[0]; ++i)
    for (uint32_t j = 0; j < x.e[1]; ++j) {
      if (!sample_row(NDIM, i, j, x.e[1])) {
        k += x.e[2];
        continue;
      }
      const T* row = field + row_base(g, x, i, j);
      for (uint32_t l = 0; l < x.e[2]; ++l, ++k) {
        const float f = regress<float, NDIM, OpRN<float>>(cf, i, j, l);
        const T v = k == kfix ? xfix : __ldg(row + l);
        E = __fadd_rn(E, fabsf(__fsub_rn(FT<T>::tofloat(v), f)));
      }
    }
  return E;
}

template <typename T, int NDIM, int B0, int B1, int B2, bool HOOK>
__device__ __forceinline__ float ereg_fast(const T* __restrict__ blk, uint64_t si, uint64_t sj, bool vec2, float4 c4,
                                           uint32_t kfix, T xfix) {
  float E = 0.0f;
  // sample rows: (i, i mod B1) in 3D; rows 1, 5, 9, ... in 2D
  constexpr int NR = NDIM == 3 ? B0 : (B1 + 2) / 4;
#pragma unroll 2
  for (int r = 0; r < NR; ++r) {
    const int i = NDIM == 3 ? r : 0;
    const int j = NDIM == 3 ? r % B1 : 4 * r + 1;
    {
      T x[B2];
      load_row<T, B2>(blk + (uint64_t)i * si + (uint64_t)j * sj, vec2, x);
      float ra, cl, cn;
      if (NDIM == 3) {
        ra = __fadd_rn(__fmul_rn(c4.x, (float)i), __fmul_rn(c4.y, (float)j));
        cl = c4.z;
        cn = c4.w;
      } else {
        ra = __fmul_rn(c4.x, (float)j);
        cl = c4.y;
        cn = c4.z;
      }
#pragma unroll
      for (int l = 0; l < B2; ++l) {
        const float f = __fadd_rn(__fadd_rn(ra, __fmul_rn(cl, (float)l)), cn);
        const T v = (HOOK && (uint32_t)((i * B1 + j) * B2 + l) == kfix) ? xfix : x[l];
        E = __fadd_rn(E, fabsf(__fsub_rn(FT<T>::tofloat(v), f)));
      }
    }
  }
  return E;
}

// The coefficients a block is selected and predicted with. Raw encoding: the fitted fp32
// values. Compact encoding: each becomes the nearest multiple of its step (a coefficient
// that cannot be stored makes the block use Lorenzo), and the selection estimate uses the
// dequantized values rounded to fp32.
template <typename T>
struct Consts;

struct CoefSel {
  float4 c4;  // for the selection estimate
  bool ok;    // regression is possible
  int k[4];   // compact encoding: the coefficient integers
};

// (the steps come from the call's State, where the bound kernel put them)
template <typename T, int NDIM>
__device__ __forceinline__ CoefSel coef_select(const Geo& g, const Ws& w, uint64_t b) {
  CoefSel r;
  r.c4 = w.coef[b];
  r.ok = (w.pflag[b] & 1) != 0;
  r.k[0] = r.k[1] = r.k[2] = r.k[3] = 0;
  if (g.enc && r.ok) {
    const float cf[4] = {r.c4.x, r.c4.y, r.c4.z, r.c4.w};
    float cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a <= NDIM; ++a) {
      if (!r.ok) break;
      r.ok = coef_to_int(cf[a], w.st->cinv[a], &r.k[a]);
      cs[a] = FT<T>::tofloat(coef_from_int<T>(r.k[a], w.st->cstep[a]));
    }
    r.c4 = make_float4(cs[0], cs[1], cs[2], cs[3]);
  }
  return r;
}

// Coefficients for prediction, with simulated memory errors applied to what is stored (the
// dtype values, or the compact encoding's integers), and the block's other error hooks. The
// compact encoding's integers are kept for the encoder here (it reads them for regression
// blocks only), so that nothing of the selection stays live through the block's pass.
template <typename T, int NDIM>
__device__ __forceinline__ void load_coefs(const Geo& g, const Ws& w, uint64_t b, const sdcsz_flip* flips,
                                           uint32_t nflips, T cT[4], Hooks& hk, CoefSel& cq, const Consts<T>& K) {
  const float4 c4 = w.coef[b];
  cT[0] = FT<T>::fromfloat(c4.x);
  cT[1] = FT<T>::fromfloat(c4.y);
  cT[2] = FT<T>::fromfloat(c4.z);
  cT[3] = FT<T>::fromfloat(c4.w);
  hk.texp = K.texp;
  hk.kp = hk.kr = hk.kfix = kNone;
  hk.bitp = hk.bitr = 0;
  hk.rewalk = false;
  if (g.enc) {
    if (nflips) {
      uint32_t lo = 0, hi = nflips;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (flips[mid].block < b) lo = mid + 1;
        else hi = mid;
      }
      for (uint32_t t = lo; t < nflips && flips[t].block == b; ++t)
        if (flips[t].site == SDCSZ_SITE_COEF && flips[t].index <= (uint64_t)NDIM)
          cq.k[flips[t].index] = (int)((uint32_t)cq.k[flips[t].index] ^ (1u << (flips[t].bit & 31)));
    }
    int* ki = static_cast<int*>(w.coefT) + 4 * b;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      cT[a] = a <= NDIM ? coef_from_int<T>(cq.k[a], w.st->cstep[a]) : T(0);
      if (a <= NDIM) ki[a] = cq.k[a];
    }
  }
  if (!nflips) return;
  uint32_t lo = 0, hi = nflips;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (flips[mid].block < b) lo = mid + 1;
    else hi = mid;
  }
  for (uint32_t t = lo; t < nflips && flips[t].block == b; ++t) {
    const sdcsz_flip f = flips[t];
    if (!g.enc && f.site == SDCSZ_SITE_COEF && f.index <= (uint64_t)NDIM) cT[f.index] = FT<T>::flip(cT[f.index], f.bit);
    if (f.site == SDCSZ_SITE_PRED && hk.kp == kNone) {
      hk.kp = (uint32_t)min(f.index, (uint64_t)kNone - 1);
      hk.bitp = f.bit;
    }
    if (f.site == SDCSZ_SITE_RECON && hk.kr == kNone) {
      hk.kr = (uint32_t)min(f.index, (uint64_t)kNone - 1);
      hk.bitr = f.bit;
    }
    if (f.site == SDCSZ_SITE_REWALK) hk.rewalk = true;
  }
}

// The coefficients of a regression block are kept for the encoder (the compact encoding's
// integers were kept by load_coefs).
template <typename T>
__device__ __forceinline__ void block_epilogue(const Ws& w, uint64_t b, bool reg, int ndim, const T cT[4],
                                               const PassRes& r, bool abft, uint8_t flag, const Geo& g) {
  if (abft) {
    w.sum_q[b] = r.sq;
    w.isum_q[b] = r.isq;
    w.sum_dc[b] = r.sdc;
  }
  w.flags[b] = flag | (reg ? 1 : 0);
  if (reg && !g.enc) {
    T* coefT = static_cast<T*>(w.coefT) + 4 * b;
    for (int a = 0; a <= ndim; ++a) coefT[a] = cT[a];
  }
}

struct Counters {
  unsigned long long unpred = 0, reg = 0, dup = 0, fix = 0, bad = 0;
  __device__ __forceinline__ void commit(State* st) {
    unpred = warp_sum(unpred);
    reg = warp_sum(reg);
    dup = warp_sum(dup);
    fix = warp_sum(fix);
    bad = warp_sum(bad);
    if ((threadIdx.x & 31) == 0) {
      if (unpred) atomicAdd(&st->n_unpred, unpred);
      if (reg) atomicAdd(&st->n_reg, reg);
      if (dup) atomicAdd(&st->dup_fixed, dup);
      if (fix) atomicAdd(&st->input_corrected, fix);
      if (bad) atomicAdd(&st->uncorrectable, bad);
    }
  }
};

// The largest |x - pred| (of the dtype) whose point certainly quantizes into the central bin and
// passes the bound check, i.e. for which quantize() returns code R and x' = pred + 0: the code
// is R iff round(round(|d| * inv2) + 1/2) < 1, i.e. round(|d| * inv2) < 1/2 - u/2 (u the ulp
// of [1/2, 1); the tie at 1 - u/2 rounds to the even 1), and the check |x - x'| <= eb then
// compares |d| itself (x' = pred, or +0 for pred = -0, leaves |x - x'| = |d|). round(d * inv2)
// never decreases with d, so one threshold D* <= eb with round(D* * inv2) below that limit
// covers every smaller |d|. Stepping down from eb takes a few ulps; -1 (never) if it does not.
template <typename T>
__device__ __forceinline__ T central_threshold(T eb, T inv2) {
  typedef typename Bitsof<T>::U U;
  const T lim = sizeof(T) == 4 ? T(0.5f - 0x1p-25f) : T(0.5 - 0x1p-54);
  T d = eb;
  for (int it = 0; it < 64 && d > T(0) && !(FT<T>::mul(d, inv2) < lim); ++it) d = Bitsof<T>::val(Bitsof<T>::raw(d) - (U)1);
  return (d > T(0) && d <= eb && FT<T>::mul(d, inv2) < lim) ? d : T(-1);
}

template <typename T>
struct Consts {
  T eb, inv2, Rh;
  T dstar;  // central_threshold(eb, inv2)
  float noise;
  int texp;  // compact encoding: truncation exponent of unpredictable values, else kNoTrunc
  __device__ __forceinline__ Consts(double ebd, const Geo& g, int ndim) {
    const uint32_t R = g.R;
    eb = (T)ebd;
    texp = g.enc ? bound_exponent<T>(eb) : kNoTrunc;
    if (sizeof(T) == 4) inv2 = (T)__double2float_rn(__ddiv_rn(1.0, __dmul_rn(2.0, ebd)));
    else inv2 = (T)__ddiv_rn(1.0, __dmul_rn(2.0, ebd));
    dstar = central_threshold<T>(eb, inv2);
    Rh = FT<T>::sub(FT<T>::fromi((int)R), T(0.5));
    // E|sum of n uniform(-1,1)| for the n = 7 / 3 / 1 Lorenzo terms (exact Irwin-Hall values)
    const float kappa = ndim == 3 ? (float)(113149.0 / 92160.0) : (ndim == 2 ? (float)(13.0 / 16.0) : 0.5f);
    noise = __fmul_rn(kappa, FT<T>::tofloat(eb));
  }
};

__device__ __forceinline__ bool block_is_full(const Geo& g, uint64_t b) {
  uint64_t c0, c1, c2;
  block_coords(g, b, c0, c1, c2);
  return (c0 + 1) * g.B[0] <= g.d[0] && (c1 + 1) * g.B[1] <= g.d[1] && (c2 + 1) * g.B[2] <= g.d[2];
}

__device__ __forceinline__ void hist_init(uint32_t* hist_s, Hist& h, const Geo& g, const Ws& w) {
  for (uint32_t q = threadIdx.x; q < kHistWindow; q += blockDim.x) hist_s[q] = 0;
  h.s = hist_s;
  h.g = w.hist;
  h.lo = g.R > kHistWindow / 2 ? g.R - kHistWindow / 2 : 0;
  h.hi = min(g.bins, h.lo + (uint32_t)kHistWindow);
}

__device__ __forceinline__ void hist_flush(uint32_t* hist_s, const Hist& h, const Ws& w) {
  __syncthreads();
  for (uint32_t q = threadIdx.x; q < h.hi - h.lo; q += blockDim.x)
    if (hist_s[q]) atomicAdd(&w.hist[h.lo + q], (unsigned long long)hist_s[q]);
}

// Algorithm 1's input check (sum_in/isum_in) after a speculative pass: returns the repaired point and
// value when a single corrupted word explains the checksum difference.
template <typename T>
__device__ __forceinline__ bool locate_input(const T* field, const Geo& g, const Box& x, unsigned long long s0,
                                             unsigned long long i0, const PassRes& r, uint32_t* kf_out, T* xf_out) {
  long long delta = 0;
  const long long m = locate_word(s0, i0, r.sw, r.isw, (unsigned long long)x.P * FT<T>::W, 0, &delta);
  if (m < 0) return false;
  const uint32_t kf = (uint32_t)(m / FT<T>::W), wi = (uint32_t)(m % FT<T>::W);
  const uint32_t lf = kf % x.e[2], tq = kf / x.e[2];
  const uint32_t jf = tq % x.e[1], i_f = tq / x.e[1];
  const T cur = field[row_base(g, x, i_f, jf) + lf];
  uint32_t wd[2] = {FT<T>::lo(cur), FT<T>::hi(cur)};
  const long long nw = (long long)wd[wi] - delta;
  if (nw < 0 || nw > 0xffffffffll) return false;
  wd[wi] = (uint32_t)nw;
  *kf_out = kf;
  *xf_out = FT<T>::from_words(wd[0], wd[1]);
  return true;
}

__device__ __forceinline__ void withdraw(const Ws& w, const Geo& g, uint64_t b, uint32_t P, const Hist& h) {
  for (uint32_t kk = 0; kk < P; ++kk) h.sub1(w.codes[code_pos(b, g.P, kk)]);
}

// One block of the generic path (runtime extents).
template <typename T, int NDIM, bool ABFT>
__device__ __forceinline__ void predict_generic_block(const T* __restrict__ field, const Geo& g, const Ws& w,
                                                      const sdcsz_flip* __restrict__ flips, uint32_t nflips,
                                                      uint64_t b, Walker<T, NDIM>& wk, const Consts<T>& K,
                                                      const Hist& h, Counters& cnt) {
  T* ustage = static_cast<T*>(w.ustage);
  const Box x = block_box(g, b);
  const uint32_t S = sample_points(NDIM, x.e);
  CoefSel cq = coef_select<T, NDIM>(g, w, b);
  bool reg = choose_reg(g, w, b, cq.ok, S, K.noise,
                        [&] { return ereg_generic<T, NDIM>(field, g, x, cq.c4, kNone, T(0)); });
  T cT[4];
  Hooks hk;
  load_coefs<T, NDIM>(g, w, b, flips, nflips, cT, hk, cq, K);
  PassRes r = reg ? generic_pass<T, NDIM, true, ABFT>(field, g, x, b, cT, wk, K.eb, K.inv2, K.Rh, w.codes, ustage,
                                                      h, hk, T(0))
                  : generic_pass<T, NDIM, false, ABFT>(field, g, x, b, cT, wk, K.eb, K.inv2, K.Rh, w.codes, ustage,
                                                       h, hk, T(0));
  uint8_t flag = 0;
  if (ABFT && (r.sw != w.sum_in[b] || r.isw != w.isum_in[b])) {
    uint32_t kf;
    T xf;
    if (locate_input<T>(field, g, x, w.sum_in[b], w.isum_in[b], r, &kf, &xf)) {
      withdraw(w, g, b, x.P, h);
      hk.kfix = kf;
      // the selection estimate and the prediction both see the repaired value
      const CoefSel cq2 = coef_select<T, NDIM>(g, w, b);
      reg = choose_reg(g, w, b, cq2.ok, S, K.noise, [&] { return ereg_generic<T, NDIM>(field, g, x, cq2.c4, kf, xf); });
      r = reg ? generic_pass<T, NDIM, true, ABFT>(field, g, x, b, cT, wk, K.eb, K.inv2, K.Rh, w.codes, ustage, h,
                                                  hk, xf)
              : generic_pass<T, NDIM, false, ABFT>(field, g, x, b, cT, wk, K.eb, K.inv2, K.Rh, w.codes, ustage, h,
                                                   hk, xf);
      ++cnt.fix;
    } else {
      ++cnt.bad;
      flag = 2;
    }
  }
  block_epilogue<T>(w, b, reg, NDIM, cT, r, ABFT, flag, g);
  cnt.unpred += r.nun;
  cnt.reg += reg;
  cnt.dup += r.dup;
}

template <typename T, int NDIM>
__device__ __forceinline__ void walker_init(Walker<T, NDIM>& wk, unsigned char* smem, const Geo& g) {
  wk.base = reinterpret_cast<T*>(smem) + threadIdx.x;
  wk.stride = blockDim.x;
  wk.B2 = g.B[2];
  wk.sr = g.B[1] * g.B[2];
}

// Generic kernel: edge blocks (or every block when `all`), any shape.
template <typename T, int NDIM, bool ABFT>
__global__ void __launch_bounds__(128) k_predict(const T* __restrict__ field, Geo g, Ws w,
                                                 const sdcsz_flip* __restrict__ flips, uint32_t nflips, int all,
                                                 uint64_t count) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t hist_s[kHistWindow];
  State* st = w.st;
  if (*(volatile unsigned int*)&st->error) return;
  Hist h;
  hist_init(hist_s, h, g, w);
  __syncthreads();
  const Consts<T> K(st->eb, g, NDIM);
  Walker<T, NDIM> wk;
  walker_init(wk, smem, g);
  Counters cnt;
  for (uint64_t it = cta_pull(&st->queue[1]); it * blockDim.x < count; it = cta_pull(&st->queue[1])) {
    const uint64_t e = it * blockDim.x + threadIdx.x;
    if (e < count)
      predict_generic_block<T, NDIM, ABFT>(field, g, w, flips, nflips, all ? e : edge_block(g, e), wk, K, h, cnt);
  }
  cnt.commit(st);
  hist_flush(hist_s, h, w);
}

// Batched generic kernel: the edge blocks (or all blocks) of every job of one dimensionality.
template <typename T, int NDIM, bool ABFT>
__global__ void __launch_bounds__(128) k_predict_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t hist_s[kHistWindow];
  __shared__ Job s_job;
  Hist h;
  Counters cnt;
  batch_loop(
      a, s_job,
      [&] {
        hist_init(hist_s, h, s_job.g, s_job.w);
        __syncthreads();
      },
      [&](uint64_t it) {
        const uint64_t e = it * blockDim.x + threadIdx.x;
        if (e < s_job.gcount) {
          const Geo& g = s_job.g;
          const Consts<T> K(s_job.w.st->eb, g, NDIM);
          Walker<T, NDIM> wk;
          walker_init(wk, smem, g);
          predict_generic_block<T, NDIM, ABFT>(static_cast<const T*>(s_job.field), g, s_job.w, nullptr, 0,
                                               s_job.fast ? edge_block(g, e) : e, wk, K, h, cnt);
        }
      },
      [&] {
        cnt.commit(s_job.w.st);
        cnt = Counters();
        hist_flush(hist_s, h, s_job.w);
      });
}

template <typename T, int NDIM, int B0, int B1, int B2, bool ABFT, bool CMP, bool HOOK, bool EDGE>
__device__ __forceinline__ PassRes fast_dispatch(bool reg, const T* blk, uint64_t si, uint64_t sj, bool vec2,
                                                 const T* cT, T* plane, const Consts<T>& K, uint32_t R, uint32_t* cptr,
                                                 T* uptr, const Hist& h, const Hooks& hk, T xfix, const uint32_t* e) {
  if (reg)
    return fast_pass<T, NDIM, B0, B1, B2, 128, true, ABFT, HOOK, CMP, EDGE>(blk, si, sj, vec2, cT, plane, K.eb, K.inv2,
                                                                       K.Rh, K.dstar, R, cptr, uptr, h, hk, xfix,
                                                                       e[0], e[1], e[2]);
  return fast_pass<T, NDIM, B0, B1, B2, 128, false, ABFT, HOOK, CMP, EDGE>(blk, si, sj, vec2, cT, plane, K.eb, K.inv2,
                                                                        K.Rh, K.dstar, R, cptr, uptr, h, hk, xfix,
                                                                        e[0], e[1], e[2]);
}

// One full block of a compile-time shape (B0 x B1 x B2, leading 1s below 3D); edge blocks
// are skipped (the generic path takes them).
// Resident CTAs of 128 threads per SM the fast kernels are compiled for (register budget).
#ifndef SDCSZ_PRED_MINB
#define SDCSZ_PRED_MINB 7
#endif

// One block with the compile-time shape B0 x B1 x B2 (leading 1s below 3D). Full blocks only,
// unless EDGE: then block b is an edge block, cut by the field boundary, walked with the same
// code and its actual extents.
template <typename T, int NDIM, int B0, int B1, int B2, bool ABFT, bool CMP, bool EDGE = false>
__device__ __forceinline__ void predict_fast_block(const T* __restrict__ field, const Geo& g, const Ws& w,
                                                   const sdcsz_flip* __restrict__ flips, uint32_t nflips, int vec2,
                                                   uint64_t b, T* plane, const Consts<T>& K, const Hist& h,
                                                   Counters& cnt) {
  T* ustage = static_cast<T*>(w.ustage);
  constexpr uint32_t P = B0 * B1 * B2;  // the layout stride (g.P)
  const uint64_t si = g.d[1] * g.d[2], sj = g.d[2];
  uint32_t e[3] = {B0, B1, B2}, Pb = P;
  const T* blk;
  Box x;
  if (EDGE) {
    x = block_box(g, b);
    e[0] = x.e[0];
    e[1] = x.e[1];
    e[2] = x.e[2];
    Pb = x.P;
    blk = field + row_base(g, x, 0, 0);
    vec2 = 0;
  } else {
    uint64_t c0, c1, c2;
    block_coords(g, b, c0, c1, c2);
    if ((c0 + 1) * B0 > g.d[0] || (c1 + 1) * B1 > g.d[1] || (c2 + 1) * B2 > g.d[2]) return;
    blk = field + (c0 * B0 * g.d[1] + c1 * B1) * g.d[2] + c2 * B2;
  }
  const uint32_t S = EDGE ? sample_points(NDIM, x.e) : (NDIM == 3 ? B0 * B2 : ((B1 + 2) / 4) * B2);
  if (!EDGE) {  // the first plane and the selection sample's rows on their way to L2
#pragma unroll
    for (int r = 0; r < B1; ++r) prefetch_l2(blk + (uint64_t)r * sj);
    if (NDIM == 3) {
#pragma unroll
      for (int i = 1; i < B0; ++i) prefetch_l2(blk + (uint64_t)i * si + (uint64_t)(i % B1) * sj);
    }
  }
  // the input checksums the walk is checked against at the end, loaded now (in flight meanwhile)
  const unsigned long long sin_ref = ABFT ? w.sum_in[b] : 0ull, isin_ref = ABFT ? w.isum_in[b] : 0ull;
  CoefSel cq = coef_select<T, NDIM>(g, w, b);
  auto ereg = [&](float4 c4, uint32_t kf, T xf) {
    if (EDGE) return ereg_generic<T, NDIM>(field, g, x, c4, kf, xf);
    if (kf != kNone) return ereg_fast<T, NDIM, B0, B1, B2, true>(blk, si, sj, vec2, c4, kf, xf);
    return ereg_fast<T, NDIM, B0, B1, B2, false>(blk, si, sj, vec2, c4, kNone, T(0));
  };
  bool reg = choose_reg(g, w, b, cq.ok, S, K.noise, [&] { return ereg(cq.c4, kNone, T(0)); });
  T cT[4];
  Hooks hk;
  load_coefs<T, NDIM>(g, w, b, flips, nflips, cT, hk, cq, K);
  uint32_t* cptr = reinterpret_cast<uint32_t*>(w.codes) + pair_index(b, P, 0);
  T* uptr = ustage + code_index(b, P, 0);
  const bool hooked = (hk.kp != kNone) || (hk.kr != kNone);
  PassRes r = hooked ? fast_dispatch<T, NDIM, B0, B1, B2, ABFT, CMP, true, EDGE>(reg, blk, si, sj, vec2, cT, plane, K, g.R,
                                                                            cptr, uptr, h, hk, T(0), e)
                     : fast_dispatch<T, NDIM, B0, B1, B2, ABFT, CMP, false, EDGE>(reg, blk, si, sj, vec2, cT, plane, K,
                                                                             g.R, cptr, uptr, h, hk, T(0), e);
  if (ABFT && (r.mm || (hk.rewalk && !hooked))) {
    // a duplicate evaluation disagreed in the unvoted walk: take the block's codes back out of
    // the histogram and walk it again with per-point voting (the same result as voting at
    // once; at least one correction counted)
    withdraw(w, g, b, Pb, h);
    r = fast_dispatch<T, NDIM, B0, B1, B2, ABFT, CMP, true, EDGE>(reg, blk, si, sj, vec2, cT, plane, K, g.R, cptr, uptr, h,
                                                             hk, T(0), e);
    r.dup = r.dup ? r.dup : 1u;
  }
  uint8_t flag = 0;
  if (ABFT && (r.sw != sin_ref || r.isw != isin_ref)) {
    if (!EDGE) x = block_box(g, b);
    uint32_t kf;
    T xf;
    if (locate_input<T>(field, g, x, sin_ref, isin_ref, r, &kf, &xf)) {
      withdraw(w, g, b, Pb, h);
      hk.kfix = kf;
      const CoefSel cq2 = coef_select<T, NDIM>(g, w, b);
      reg = choose_reg(g, w, b, cq2.ok, S, K.noise, [&] { return ereg(cq2.c4, kf, xf); });
      r = fast_dispatch<T, NDIM, B0, B1, B2, ABFT, CMP, true, EDGE>(reg, blk, si, sj, vec2, cT, plane, K, g.R, cptr, uptr, h,
                                                               hk, xf, e);
      ++cnt.fix;
    } else {
      ++cnt.bad;
      flag = 2;
    }
  }
  block_epilogue<T>(w, b, reg, NDIM, cT, r, ABFT, flag, g);
  cnt.unpred += r.nun;
  cnt.reg += reg;
  cnt.dup += r.dup;
}

// Edge blocks of a field whose full blocks take the fast kernel: the same compile-time
// walk with runtime extents, one thread per edge block (compact enumeration).
template <typename T, int NDIM, int B0, int B1, int B2, bool ABFT, bool CMP>
__global__ void __launch_bounds__(128, SDCSZ_PRED_MINB) k_predict_edge(const T* __restrict__ field, Geo g, Ws w,
                                                      const sdcsz_flip* __restrict__ flips, uint32_t nflips,
                                                      uint64_t count) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t hist_s[kHistWindow];
  State* st = w.st;
  if (*(volatile unsigned int*)&st->error) return;
  Hist h;
  hist_init(hist_s, h, g, w);
  __syncthreads();
  const Consts<T> K(st->eb, g, NDIM);
  T* plane = reinterpret_cast<T*>(smem) + threadIdx.x;
  Counters cnt;
  for (uint64_t it = cta_pull(&st->queue[1]); it * blockDim.x < count; it = cta_pull(&st->queue[1])) {
    const uint64_t e = it * blockDim.x + threadIdx.x;
    if (e < count)
      predict_fast_block<T, NDIM, B0, B1, B2, ABFT, CMP, true>(field, g, w, flips, nflips, 0, edge_block(g, e), plane, K,
                                                          h, cnt);
  }
  cnt.commit(st);
  hist_flush(hist_s, h, w);
}

// Fast kernel: full blocks of a compile-time shape.
template <typename T, int NDIM, int B0, int B1, int B2, bool ABFT, bool CMP>
__global__ void __launch_bounds__(128, SDCSZ_PRED_MINB) k_predict_fast(const T* __restrict__ field, Geo g, Ws w,
                                                      const sdcsz_flip* __restrict__ flips, uint32_t nflips,
                                                      int vec2) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t hist_s[kHistWindow];
  State* st = w.st;
  if (*(volatile unsigned int*)&st->error) return;
  Hist h;
  hist_init(hist_s, h, g, w);
  __syncthreads();
  const Consts<T> K(st->eb, g, NDIM);
  T* plane = reinterpret_cast<T*>(smem) + threadIdx.x;
  Counters cnt;
  for (uint64_t it = cta_pull(&st->queue[0]); it * blockDim.x < g.nb; it = cta_pull(&st->queue[0])) {
    const uint64_t b = it * blockDim.x + threadIdx.x;
    if (b < g.nb) predict_fast_block<T, NDIM, B0, B1, B2, ABFT, CMP>(field, g, w, flips, nflips, vec2, b, plane, K, h, cnt);
  }
  cnt.commit(st);
  hist_flush(hist_s, h, w);
}

// Batched fast kernel: the full blocks of every job with this block shape.
template <typename T, int NDIM, int B0, int B1, int B2, bool ABFT, bool CMP>
__global__ void __launch_bounds__(128, SDCSZ_PRED_MINB) k_predict_fast_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t hist_s[kHistWindow];
  __shared__ Job s_job;
  Hist h;
  Counters cnt;
  T* plane = reinterpret_cast<T*>(smem) + threadIdx.x;
  batch_loop(
      a, s_job,
      [&] {
        hist_init(hist_s, h, s_job.g, s_job.w);
        __syncthreads();
      },
      [&](uint64_t it) {
        const uint64_t b = it * blockDim.x + threadIdx.x;
        if (b < s_job.g.nb) {
          const Consts<T> K(s_job.w.st->eb, s_job.g, NDIM);
          predict_fast_block<T, NDIM, B0, B1, B2, ABFT, CMP>(static_cast<const T*>(s_job.field), s_job.g, s_job.w,
                                                        nullptr, 0, s_job.vec2, b, plane, K, h, cnt);
        }
      },
      [&] {
        cnt.commit(s_job.w.st);
        cnt = Counters();
        hist_flush(hist_s, h, s_job.w);
      });
}

}  // namespace
}  // namespace kpred
}  // namespace sdcsz

#include "predict_wave.cuh"

namespace sdcsz {
namespace kpred {
namespace {

// ---------------------------------------------------------------- launch
// Shared memory the one-thread-per-block kernels may ask for (128 threads' Lorenzo planes).
constexpr size_t kLanePlaneSmemMax = 200 * 1024;

template <class K>
inline void launch_persistent(K kern, uint32_t threads, size_t smem, uint64_t nb, const Launch& L, dim3* grid_out) {
  const int occ = occupancy(reinterpret_cast<const void*>(kern), (int)threads, smem);
  const uint64_t need = (nb + threads - 1) / threads;
  *grid_out = dim3((unsigned)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)occ * L.sms)));
}

template <typename T, int NDIM, bool ABFT>
void run_generic(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips, bool all,
                 const Launch& L) {
  const uint32_t per = walker_slots(g.ndim, g.B) * sizeof(T);
  uint32_t threads = 128;
  while (threads > 32 && (size_t)per * threads > 160 * 1024) threads >>= 1;
  const size_t smem = (size_t)per * threads;
  auto kern = k_predict<T, NDIM, ABFT>;
  const uint64_t count = all ? g.nb : edge_count(g);
  if (!count) return;
  dim3 grid;
  launch_persistent(kern, threads, smem, count, L, &grid);
  kern<<<grid, threads, smem, L.stream>>>(static_cast<const T*>(field), g, w, flips, nflips, all ? 1 : 0, count);
  note_launch();
}

template <typename T, int NDIM, int B0, int B1, int B2, bool ABFT, bool CMP>
void run_fast(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
              const Launch& L) {
  const size_t smem = (NDIM == 3) ? (size_t)B1 * B2 * 128 * sizeof(T) : 0;
  auto kern = k_predict_fast<T, NDIM, B0, B1, B2, ABFT, CMP>;
  dim3 grid;
  launch_persistent(kern, 128, smem, g.nb, L, &grid);
  const bool vec2 = (B2 % 2 == 0) && (g.d[2] % 2 == 0) &&
                    (reinterpret_cast<uintptr_t>(field) % (2 * sizeof(T)) == 0);
  kern<<<grid, 128, smem, L.stream>>>(static_cast<const T*>(field), g, w, flips, nflips, vec2 ? 1 : 0);
  note_launch();
}

// Cube blocks of edge B (10, 12, 16) by the wavefront kernel, G blocks per CTA: the full
// blocks (edge = false), or the blocks cut by the field boundary (edge = true, their compact
// enumeration, on the second work queue).
template <typename T, int B, int G, bool ABFT, bool CMP>
void run_wave(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
              const Launch& L, bool edge) {
  typedef WaveCfg<T, B, G> C;
  auto kern = k_predict_wave<T, B, G, ABFT, CMP>;
  const uint64_t count = edge ? edge_count(g) : g.nb;
  if (!count) return;
  const uint64_t ngroups = (count + G - 1) / G;
  dim3 grid;
  launch_persistent(kern, C::NT, C::SMEM, ngroups * C::NT, L, &grid);
  kern<<<grid, C::NT, C::SMEM, L.stream>>>(static_cast<const T*>(field), g, w, flips, nflips, edge ? 1 : 0, count);
  note_launch();
}

template <typename T, int NDIM, int B0, int B1, int B2, bool ABFT, bool CMP>
void run_edge(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
              const Launch& L) {
  const uint64_t count = edge_count(g);
  if (!count) return;
  const size_t smem = (NDIM == 3) ? (size_t)B1 * B2 * 128 * sizeof(T) : 0;
  if (smem > kLanePlaneSmemMax) {  // 128 threads' planes would not fit: the generic walk
    run_generic<T, NDIM, ABFT>(field, g, w, flips, nflips, false, L);
    return;
  }
  auto kern = k_predict_edge<T, NDIM, B0, B1, B2, ABFT, CMP>;
  dim3 grid;
  launch_persistent(kern, 128, smem, count, L, &grid);
  kern<<<grid, 128, smem, L.stream>>>(static_cast<const T*>(field), g, w, flips, nflips, count);
  note_launch();
}

template <typename T, bool ABFT, bool CMP>
void try_edge(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
              const Launch& L) {
  if (g.ndim == 3) {
    switch (g.B[2]) {
      case 4: run_edge<T, 3, 4, 4, 4, ABFT, CMP>(field, g, w, flips, nflips, L); break;
      case 6: run_edge<T, 3, 6, 6, 6, ABFT, CMP>(field, g, w, flips, nflips, L); break;
      case 8: run_edge<T, 3, 8, 8, 8, ABFT, CMP>(field, g, w, flips, nflips, L); break;
      case 10: run_edge<T, 3, 10, 10, 10, ABFT, CMP>(field, g, w, flips, nflips, L); break;
      case 12: run_wave<T, 12, wave_group_blocks(12), ABFT, CMP>(field, g, w, flips, nflips, L, true); break;
      case 16: run_wave<T, 16, wave_group_blocks(16), ABFT, CMP>(field, g, w, flips, nflips, L, true); break;
      default: break;
    }
  } else if (g.ndim == 2) {
    switch (g.B[2]) {
      case 8: run_edge<T, 2, 1, 8, 8, ABFT, CMP>(field, g, w, flips, nflips, L); break;
      case 12: run_edge<T, 2, 1, 12, 12, ABFT, CMP>(field, g, w, flips, nflips, L); break;
      case 16: run_edge<T, 2, 1, 16, 16, ABFT, CMP>(field, g, w, flips, nflips, L); break;
      default: break;
    }
  }
}

// Shapes with a fast path: cubes 4..16 in 3D, squares 8/12/16 in 2D.
inline bool has_fast(const Geo& g) {
  if (g.ndim == 3 && g.B[0] == g.B[1] && g.B[1] == g.B[2])
    return g.B[2] == 4 || g.B[2] == 6 || g.B[2] == 8 || g.B[2] == 10 || g.B[2] == 12 || g.B[2] == 16;
  if (g.ndim == 2 && g.B[1] == g.B[2]) return g.B[2] == 8 || g.B[2] == 12 || g.B[2] == 16;
  return false;
}

template <typename T, bool ABFT, bool CMP>
bool try_fast(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
              const Launch& L) {
  if (g.ndim == 3 && g.B[0] == g.B[1] && g.B[1] == g.B[2]) {
    switch (g.B[2]) {
      case 4: run_fast<T, 3, 4, 4, 4, ABFT, CMP>(field, g, w, flips, nflips, L); return true;
      case 6: run_fast<T, 3, 6, 6, 6, ABFT, CMP>(field, g, w, flips, nflips, L); return true;
      case 8: run_fast<T, 3, 8, 8, 8, ABFT, CMP>(field, g, w, flips, nflips, L); return true;
      case 10: run_fast<T, 3, 10, 10, 10, ABFT, CMP>(field, g, w, flips, nflips, L); return true;
      case 12: run_wave<T, 12, wave_group_blocks(12), ABFT, CMP>(field, g, w, flips, nflips, L, false); return true;
      case 16: run_wave<T, 16, wave_group_blocks(16), ABFT, CMP>(field, g, w, flips, nflips, L, false); return true;
      default: return false;
    }
  }
  if (g.ndim == 2 && g.B[1] == g.B[2]) {
    switch (g.B[2]) {
      case 8: run_fast<T, 2, 1, 8, 8, ABFT, CMP>(field, g, w, flips, nflips, L); return true;
      case 12: run_fast<T, 2, 1, 12, 12, ABFT, CMP>(field, g, w, flips, nflips, L); return true;
      case 16: run_fast<T, 2, 1, 16, 16, ABFT, CMP>(field, g, w, flips, nflips, L); return true;
      default: return false;
    }
  }
  return false;
}

template <typename T, bool ABFT, bool CMP>
void launch_predict_t(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                      const Launch& L) {
  // shapes with a fast path: edge blocks on the side stream with the same compile-time walk,
  // concurrently with the full blocks; other shapes: the generic kernel for every block
  if (has_fast(g)) {
    Fork fk(L);
    try_edge<T, ABFT, CMP>(field, g, w, flips, nflips, fk.side_launch(L));
    try_fast<T, ABFT, CMP>(field, g, w, flips, nflips, L);
    fk.join();
  } else if (g.ndim == 3) {
    run_generic<T, 3, ABFT>(field, g, w, flips, nflips, true, L);
  } else if (g.ndim == 2) {
    run_generic<T, 2, ABFT>(field, g, w, flips, nflips, true, L);
  } else {
    run_generic<T, 1, ABFT>(field, g, w, flips, nflips, true, L);
  }
}

// ---------------------------------------------------------------- batched launches
template <typename T, int NDIM, int B0, int B1, int B2, bool ABFT, bool CMP>
void batch_fast(const BatchArgs& a, const Launch& L) {
  const size_t smem = (NDIM == 3) ? (size_t)B1 * B2 * 128 * sizeof(T) : 0;
  auto kern = k_predict_fast_batch<T, NDIM, B0, B1, B2, ABFT, CMP>;
  dim3 grid;
  launch_persistent(kern, 128, smem, a.start[a.n] * 128, L, &grid);
  kern<<<grid, 128, smem, L.stream>>>(a);
  note_launch();
}

// Batched wavefront kernel: items are groups of G blocks (wave_groups).
template <typename T, int B, int G, bool ABFT, bool CMP>
void batch_wave(const BatchArgs& a, const Launch& L) {
  static_assert(G == wave_group_blocks(B), "the launch plan counts groups of this size");
  typedef WaveCfg<T, B, G> C;
  auto kern = k_predict_wave_batch<T, B, G, ABFT, CMP>;
  dim3 grid;
  launch_persistent(kern, C::NT, C::SMEM, a.start[a.n] * C::NT, L, &grid);
  kern<<<grid, C::NT, C::SMEM, L.stream>>>(a);
  note_launch();
}

template <typename T, bool ABFT, bool CMP>
bool batch_fast_shape(int ndim, uint32_t B, const BatchArgs& a, const Launch& L) {
  if (ndim == 3) {
    switch (B) {
      case 4: batch_fast<T, 3, 4, 4, 4, ABFT, CMP>(a, L); return true;
      case 6: batch_fast<T, 3, 6, 6, 6, ABFT, CMP>(a, L); return true;
      case 8: batch_fast<T, 3, 8, 8, 8, ABFT, CMP>(a, L); return true;
      case 10: batch_fast<T, 3, 10, 10, 10, ABFT, CMP>(a, L); return true;
      case 12: batch_wave<T, 12, wave_group_blocks(12), ABFT, CMP>(a, L); return true;
      case 16: batch_wave<T, 16, wave_group_blocks(16), ABFT, CMP>(a, L); return true;
      default: return false;
    }
  }
  if (ndim == 2) {
    switch (B) {
      case 8: batch_fast<T, 2, 1, 8, 8, ABFT, CMP>(a, L); return true;
      case 12: batch_fast<T, 2, 1, 12, 12, ABFT, CMP>(a, L); return true;
      case 16: batch_fast<T, 2, 1, 16, 16, ABFT, CMP>(a, L); return true;
      default: return false;
    }
  }
  return false;
}

template <typename T, int NDIM, bool ABFT>
void batch_generic(const BatchArgs& a, uint32_t threads, size_t smem, const Launch& L) {
  auto kern = k_predict_batch<T, NDIM, ABFT>;
  dim3 grid;
  launch_persistent(kern, threads, smem, a.start[a.n] * threads, L, &grid);
  kern<<<grid, threads, smem, L.stream>>>(a);
  note_launch();
}

template <typename T, bool ABFT>
void batch_generic_dim(int ndim, const BatchArgs& a, uint32_t threads, size_t smem, const Launch& L) {
  if (ndim == 3) batch_generic<T, 3, ABFT>(a, threads, smem, L);
  else if (ndim == 2) batch_generic<T, 2, ABFT>(a, threads, smem, L);
  else batch_generic<T, 1, ABFT>(a, threads, smem, L);
}

}  // namespace
}  // namespace kpred
}  // namespace sdcsz
