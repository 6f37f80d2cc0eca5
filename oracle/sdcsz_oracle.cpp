// Oracle for the SDC-resilient, independent-block SZ compressor.
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow, single-threaded CPU restatement of
// the paper's method, used by tests/, by __graft_entry__.smoke() and by bench.py's CPU
// baseline leg to check and time the CUDA library. The product path never links or calls it,
// and it shares no code, header, table or constant generator with the CUDA sources.
//
// Paper: "SDC Resilient Error-bounded Lossy Compressor" (Li, Di, Zhao, Liang, Chen,
// Cappello; arXiv 2010.03144).
//   Sec. 3.1   SZ stages: prediction (improved Lorenzo or linear regression per block),
//              linear-scaling quantization, Huffman coding (lossless Zstd stage left out).
//   Sec. 3.2   ABFT checksum pair sum = sum a[i], isum = sum i*a[i]; a single corrupted
//              element is located at j = (isum1 - isum0) / (sum1 - sum0).
//   Sec. 3.3   Error model: at most one error per block per run; checksums error free.
//   Sec. 4.1.2 The prediction / quantization / reconstruction / double-check loop.
//   Sec. 5.1   Independent blocks, per-block compressed size recorded (random access).
//   Alg. 1     Fault-tolerant compression; Alg. 2 fault-tolerant decompression.
//   Sec. 5.4   Checksums over the bit patterns (u32 words widened to u64; fp64 = 2 words).
//   Sec. 5.5   CR-decrease bound for unprotected regression/sampling.
//
// Where the paper is silent the oracle takes one fixed reading, which the CUDA library
// implements identically:
//   * partial edge blocks use their actual extents; local order is row-major;
//   * value-range bound eb = (T)(e * ((double)max - (double)min)) over finite values;
//   * checksum weights are 1-based so every word contributes to isum;
//   * regression and the sampled estimates read the input as it is when compression starts
//     (simulated input errors land after them); the input is verified/corrected before any
//     value is predicted, so a repaired block compresses as the error-free one;
//   * regression: closed-form least squares on the block grid in fp32, sequential sums;
//   * selection: the sample is a set of whole rows (one diagonal row per plane in 3D, every
//     fourth row in 2D); E_lor adds kappa*eb per sample point (kappa exact, see below);
//   * duplication recomputes once more on a mismatch and keeps the third result;
//   * the histogram is taken as the codes are produced (before the bin-array window that
//     the code checksums protect);
//   * Huffman: (weight, creation order) tie-break, lengths limited to 24 bits by the
//     JPEG (ITU T.81 Annex K.3) adjustment, canonical codes, MSB-first bit order;
//   * the byte layout of the stream;
//   * the compact encoding (SZ's own coefficient and unpredictable-value encodings, kept
//     block-local): regression coefficients as integer multiples of a step tied to the bound
//     (slopes eb/(16 B_a), intercept eb/16, round half away from zero in double), written
//     as length-prefixed zigzag integers at the head of the block's payload; unpredictable
//     values truncated to the mantissa bits the bound needs and written right after their
//     code 0;
//   * the lossless stage (Algorithm 1's final step, Zstd in the paper) is an order-0 range
//     asymmetric numeral system coder of our own over the bytes after the block tables
//     (sum_dc, coefficients, unpredictable values, payload), in independent 16 KiB chunks
//     of 32 interleaved states.
// The predictor-selection estimate (kappa, sample set) only changes the compression ratio
// (Sec. 4.1.1); it is pinned by hand-listed sample rows, exact rational kappa values and
// integer blocks whose estimates are exact (tests/test_oracle_selection.py).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <queue>
#include <type_traits>
#include <vector>

extern "C" {

typedef struct {
  uint32_t ndim;        // 1..3
  uint32_t dtype;       // 0 = float32, 1 = float64
  uint64_t dims[3];     // slowest first, C order
  uint32_t block[3];    // block edge per dim
  uint32_t eb_mode;     // 0 = absolute, 1 = value-range relative
  double eb;            // user error bound e
  uint32_t quant_bins;  // even, 2..65536
  uint32_t abft;        // 1 = fault tolerant (ftrsz), 0 = plain independent blocks (rsz)
  uint32_t predictor;   // 0 = select per block, 1 = Lorenzo only, 2 = regression only
  uint32_t encoding;    // bit 0: compact coefficient / unpredictable encoding; bit 1: lossless stage
} orc_params;

typedef struct {
  uint64_t blocks, regression_blocks, unpredictable_points, compressed_bytes;
  uint64_t input_corrected, codes_corrected, dup_mismatch_corrected;
  uint64_t decomp_reexec_corrected, uncorrectable_blocks;
  uint64_t bound_violations;
  double eb_abs;
  double max_abs_err;
} orc_report;

// One simulated soft error. Sites:
//   1 input word  (index = global u32 word of the field; hits after the input checksums)
//   2 code        (block, index = local point; hits after the codes are checksummed)
//   3 coefficient (block, index = coefficient; hits after selection, before prediction)
//   4 prediction  (block, index = local point; transient error in the first evaluation)
//   5 reconstruct (block, index = local point; transient error in the first evaluation)
//   6 decompress  (block, index = local point; transient error in the first decompression)
typedef struct {
  uint32_t site, bit;
  uint64_t block, index;
} orc_flip;

}  // extern "C"

namespace {

enum { OK = 0, EINVAL_ = -1, ECAPACITY = -2, EFORMAT = -3, ESDC = -4 };
enum { SITE_INPUT = 1, SITE_CODE = 2, SITE_COEF = 3, SITE_PRED = 4, SITE_RECON = 5, SITE_DECOMP = 6 };

constexpr uint32_t kMaxLen = 24;   // longest Huffman code (bits)
constexpr uint64_t kGroup = 256;   // blocks per random-access group
constexpr uint32_t kHeader = 128;  // header bytes

// ---------------------------------------------------------------- geometry (Sec. 5.1)
struct Geom {
  int ndim = 0;
  int dtype = 0;
  uint64_t d[3] = {1, 1, 1};   // padded to 3D, leading 1s
  uint32_t B[3] = {1, 1, 1};
  uint64_t nbd[3] = {1, 1, 1};
  uint64_t nb = 0, N = 0;
  uint32_t P = 0;              // points in a full block
};

bool make_geom(const orc_params* p, Geom* g) {
  if (p->ndim < 1 || p->ndim > 3 || p->dtype > 1) return false;
  g->ndim = (int)p->ndim;
  g->dtype = (int)p->dtype;
  const int off = 3 - g->ndim;
  uint64_t N = 1, nb = 1, P = 1;
  for (int a = 0; a < g->ndim; ++a) {
    uint64_t n = p->dims[a];
    uint32_t b = p->block[a];
    if (n > (1ull << 40)) return false;
    if (b < 2) return false;
    if (g->ndim == 3 && b > 16) return false;
    if (g->ndim == 2 && b > 64) return false;
    if (g->ndim == 1 && b > 4096) return false;
    g->d[off + a] = n;
    g->B[off + a] = b;
    g->nbd[off + a] = (n + b - 1) / b;
    N *= n;
    nb *= g->nbd[off + a];
    P *= b;
  }
  if (P > 4096 || N > (1ull << 40)) return false;
  g->N = N;
  g->nb = nb;
  g->P = (uint32_t)P;
  return true;
}

void block_box(const Geom& g, uint64_t b, uint64_t org[3], uint32_t ext[3]) {
  uint64_t c2 = b % g.nbd[2];
  uint64_t t = b / g.nbd[2];
  uint64_t c1 = t % g.nbd[1];
  uint64_t c0 = t / g.nbd[1];
  uint64_t c[3] = {c0, c1, c2};
  for (int a = 0; a < 3; ++a) {
    org[a] = c[a] * g.B[a];
    uint64_t rem = g.d[a] - org[a];
    ext[a] = (uint32_t)std::min<uint64_t>(g.B[a], rem);
  }
}

uint64_t global_index(const Geom& g, const uint64_t org[3], uint32_t i, uint32_t j, uint32_t l) {
  return ((org[0] + i) * g.d[1] + (org[1] + j)) * g.d[2] + (org[2] + l);
}

// ---------------------------------------------------------------- bit patterns (Sec. 5.4)
template <typename T> struct Bits;
template <> struct Bits<float> {
  static constexpr int kWords = 1;
  static void words(float x, uint32_t w[2]) { std::memcpy(&w[0], &x, 4); }
  static float from_words(const uint32_t w[2]) { float x; std::memcpy(&x, &w[0], 4); return x; }
  static bool same(float a, float b) { uint32_t u, v; std::memcpy(&u, &a, 4); std::memcpy(&v, &b, 4); return u == v; }
  static float flip(float x, uint32_t bit) { uint32_t u; std::memcpy(&u, &x, 4); u ^= (1u << (bit & 31)); std::memcpy(&x, &u, 4); return x; }
};
template <> struct Bits<double> {
  static constexpr int kWords = 2;
  static void words(double x, uint32_t w[2]) {
    uint64_t u; std::memcpy(&u, &x, 8); w[0] = (uint32_t)u; w[1] = (uint32_t)(u >> 32);  // low word first
  }
  static double from_words(const uint32_t w[2]) {
    uint64_t u = (uint64_t)w[0] | ((uint64_t)w[1] << 32); double x; std::memcpy(&x, &u, 8); return x;
  }
  static bool same(double a, double b) { uint64_t u, v; std::memcpy(&u, &a, 8); std::memcpy(&v, &b, 8); return u == v; }
  static double flip(double x, uint32_t bit) { uint64_t u; std::memcpy(&u, &x, 8); u ^= (1ull << (bit & 63)); std::memcpy(&x, &u, 8); return x; }
};

// Sec. 3.2 / Sec. 5.4: sum = sum of words, isum = sum of (m+1)*word_m, both modulo 2^64.
void checksum_words(const uint32_t* w, uint64_t n, uint64_t* sum, uint64_t* isum) {
  uint64_t s = 0, is = 0;
  for (uint64_t m = 0; m < n; ++m) {
    s += (uint64_t)w[m];
    is += (uint64_t)(m + 1) * (uint64_t)w[m];
  }
  *sum = s;
  *isum = is;
}

// Sec. 3.2: a single changed element j changes sum by delta and isum by (j+1)*delta.
// Returns 0 when clean, 1 when one word was located and repaired, 2 when the difference
// is not explained by a single corrupted word (outside the error model of Sec. 3.3).
int locate_and_repair(uint32_t* w, uint64_t n, uint64_t sum0, uint64_t isum0, uint64_t maxval) {
  uint64_t s1, is1;
  checksum_words(w, n, &s1, &is1);
  int64_t ds = (int64_t)(s1 - sum0);
  int64_t dis = (int64_t)(is1 - isum0);
  if (ds == 0 && dis == 0) return 0;
  if (ds == 0) return 2;
  if (dis % ds != 0) return 2;
  int64_t pos = dis / ds;  // = m + 1
  if (pos < 1 || (uint64_t)pos > n) return 2;
  int64_t fixed = (int64_t)w[pos - 1] - ds;
  if (fixed < 0 || (uint64_t)fixed > maxval) return 2;
  w[pos - 1] = (uint32_t)fixed;
  return 1;
}

// ---------------------------------------------------------------- predictors (Sec. 3.1)
// Improved Lorenzo predictor on block-local values d (row-major, extents e), with zero
// for neighbours outside the block (independent blocks, Sec. 5.1). The operand order is
// fixed so that every implementation rounds identically: the neighbours in the previous
// row and plane first, the previous point of the same row last.
template <typename T>
T lorenzo(const T* d, const uint32_t e[3], int ndim, uint32_t i, uint32_t j, uint32_t l) {
  auto at = [&](long ii, long jj, long ll) -> T {
    if (ii < 0 || jj < 0 || ll < 0) return (T)0;
    return d[((uint64_t)ii * e[1] + (uint64_t)jj) * e[2] + (uint64_t)ll];
  };
  long I = i, J = j, L = l;
  if (ndim == 3) {
    T s = at(I - 1, J, L) + at(I, J - 1, L);
    s = s - at(I - 1, J - 1, L);
    s = s - at(I - 1, J, L - 1);
    s = s - at(I, J - 1, L - 1);
    s = s + at(I - 1, J - 1, L - 1);
    s = s + at(I, J, L - 1);
    return s;
  }
  if (ndim == 2) {
    T s = at(0, J - 1, L) - at(0, J - 1, L - 1);
    s = s + at(0, J, L - 1);
    return s;
  }
  return at(0, 0, L - 1);
}

// Linear regression predictor: ((b0*c0 + b1*c1) + b2*c2) + b_n over the block's own
// coordinates (Sec. 3.1; at most 4 coefficients in 3D, Sec. 4.2.2).
template <typename T>
T regress(const T* coef, int ndim, const uint32_t coord3[3]) {
  const int off = 3 - ndim;
  T acc = coef[0] * (T)coord3[off];
  for (int a = 1; a < ndim; ++a) acc = acc + coef[a] * (T)coord3[off + a];
  return acc + coef[ndim];
}

// Closed-form least-squares fit on the regular block grid, in fp32 (Algorithm 1, regression).
// Slopes decouple on a full grid: b_a = sum x*(c_a - ctr_a) / sum (c_a - ctr_a)^2, and the
// intercept makes the fit pass through the mean. Sums are taken per row along the fastest
// axis first (r0 = sum x, rl = sum x*(l - ctr_l), in increasing l), then the row sums are
// added into the block sums in increasing row order (S0 += r0, S_l += rl, S_a += r0*(c_a -
// ctr_a) for the slower axes, whose coordinate is constant along a row).
template <typename T>
bool regression_coefficients(const T* v, const uint32_t e[3], int ndim, float coef[4]) {
  const int off = 3 - ndim;
  const uint64_t P = (uint64_t)e[0] * e[1] * e[2];
  float ctr[3] = {0.0f, 0.0f, 0.0f}, D[3] = {0.0f, 0.0f, 0.0f};
  for (int a = 0; a < ndim; ++a) {
    uint32_t ed = e[off + a];
    ctr[a] = 0.5f * (float)(ed - 1);
    D[a] = (float)((double)P * ((double)ed * (double)ed - 1.0) / 12.0);
  }
  float S0 = 0.0f, S[3] = {0.0f, 0.0f, 0.0f};
  uint64_t k = 0;
  const int fast = ndim - 1;  // index of the fastest axis among the active ones
  for (uint32_t i = 0; i < e[0]; ++i)
    for (uint32_t j = 0; j < e[1]; ++j) {
      float r0 = 0.0f, rl = 0.0f;
      for (uint32_t l = 0; l < e[2]; ++l, ++k) {
        float xr = (float)v[k];
        r0 = r0 + xr;
        rl = rl + xr * ((float)l - ctr[fast]);
      }
      uint32_t c3[3] = {i, j, 0};
      S0 = S0 + r0;
      S[fast] = S[fast] + rl;
      for (int a = 0; a < fast; ++a) S[a] = S[a] + r0 * ((float)c3[off + a] - ctr[a]);
    }
  for (int a = 0; a < ndim; ++a) coef[a] = (e[off + a] > 1) ? S[a] / D[a] : 0.0f;
  float mean = S0 / (float)P;
  float acc = coef[0] * ctr[0];
  for (int a = 1; a < ndim; ++a) acc = acc + coef[a] * ctr[a];
  coef[ndim] = mean - acc;
  for (int a = 0; a <= ndim; ++a)
    if (!std::isfinite(coef[a])) return false;
  return true;
}

// The sample of Algorithm 1's "sample and estimate" step: whole rows along the fastest axis. 3D: one row per plane, the
// "diagonal" rows (i, i mod e1); 2D: every fourth row starting with row 1 (rows 1, 5, 9, ...);
// 1D: the whole block.
bool sample_row(int ndim, uint32_t i, uint32_t j, const uint32_t e[3]) {
  if (ndim == 3) return j == i % e[1];
  if (ndim == 2) return (j & 3u) == 1u;
  return true;
}

uint64_t sample_points(int ndim, const uint32_t e[3]) {
  uint64_t n = 0;
  for (uint32_t i = 0; i < e[0]; ++i)
    for (uint32_t j = 0; j < e[1]; ++j)
      if (sample_row(ndim, i, j, e)) n += e[2];
  return n;
}

// Selection estimates (Algorithm 1), in fp32 over the sample points in local order:
// E_reg = sum |x - f_reg|, E_lor = sum |x - Lorenzo(original values)|.
template <typename T>
void selection_estimates(const T* v, const uint32_t e[3], int ndim, const float coef[4], float* Ereg_out,
                         float* Elor_out) {
  const uint64_t P = (uint64_t)e[0] * e[1] * e[2];
  std::vector<float> xr(P);
  for (uint64_t k = 0; k < P; ++k) xr[k] = (float)v[k];
  float Ereg = 0.0f, Elor = 0.0f;
  uint64_t k = 0;
  for (uint32_t i = 0; i < e[0]; ++i)
    for (uint32_t j = 0; j < e[1]; ++j)
      for (uint32_t l = 0; l < e[2]; ++l, ++k) {
        if (!sample_row(ndim, i, j, e)) continue;
        uint32_t c3[3] = {i, j, l};
        float f = regress<float>(coef, ndim, c3);
        Ereg = Ereg + std::fabs(xr[k] - f);
        float L = lorenzo<float>(xr.data(), e, ndim, i, j, l);
        Elor = Elor + std::fabs(xr[k] - L);
      }
  *Ereg_out = Ereg;
  *Elor_out = Elor;
}

// Algorithm 1's indicator: the predictor with the smaller estimated error. E_lor gets the expected
// effect of predicting from reconstructed instead of original neighbours: kappa*eb per point,
// kappa = E|sum of n uniform(-eb,eb)| / eb for the n = 1, 3, 7 Lorenzo terms of 1D/2D/3D, the
// exact Irwin-Hall expectations 1/2, 13/16 and 113149/92160, rounded to fp32.
bool select_regression(float Ereg, float Elor, uint64_t S, int ndim, float ebf) {
  static const float kappa[4] = {0.0f, (float)(1.0 / 2.0), (float)(13.0 / 16.0), (float)(113149.0 / 92160.0)};
  float noise = kappa[ndim] * ebf;
  float total = Elor + (float)S * noise;
  return Ereg < total;
}

// ---------------------------------------------------------------- compact encoding
// Steps of the coefficient quantization for an absolute bound E (the dtype value): slope a
// moves the prediction by at most (B_a - 1) * step_a / 2 across the block and the intercept by
// step / 2, so the rounded coefficients shift a prediction by less than eb / 8 in total.
struct CoefSteps {
  double step[4], inv[4];
};

CoefSteps coef_steps(const Geom& g, double E) {
  CoefSteps q;
  const int off = 3 - g.ndim;
  for (int a = 0; a < 4; ++a) q.step[a] = q.inv[a] = 0.0;
  for (int a = 0; a < g.ndim; ++a) {
    const double d = 16.0 * (double)g.B[off + a];
    q.step[a] = E / d;
    q.inv[a] = d / E;
  }
  q.step[g.ndim] = E / 16.0;
  q.inv[g.ndim] = 16.0 / E;
  return q;
}

// Nearest multiple of the step (halves away from zero); false when it is not finite or not
// below 2^30 steps, which makes the block use Lorenzo.
bool quantize_coef(float c, double inv, int32_t* k) {
  const double t = (double)c * inv;
  if (!(std::fabs(t) < 1073741824.0)) return false;
  const double m = std::floor(std::fabs(t) + 0.5);
  *k = (int32_t)(t < 0.0 ? -m : m);
  return true;
}

template <typename T> T dequantize_coef(int32_t k, double step) { return (T)((double)k * step); }

// Bit fields of the dtype: mantissa bits, exponent bits, exponent bias.
template <typename T> struct Fmt;
template <> struct Fmt<float> {
  typedef uint32_t U;
  static constexpr int M = 23, E = 8, BIAS = 127;
};
template <> struct Fmt<double> {
  typedef uint64_t U;
  static constexpr int M = 52, E = 11, BIAS = 1023;
};

template <typename T> typename Fmt<T>::U raw_bits(T x) {
  typename Fmt<T>::U u;
  std::memcpy(&u, &x, sizeof(T));
  return u;
}

template <typename T> T from_raw(typename Fmt<T>::U u) {
  T x;
  std::memcpy(&x, &u, sizeof(T));
  return x;
}

// floor(log2(eb)) of a normal bound
template <typename T> int bound_exponent(T eb) {
  return (int)((raw_bits<T>(eb) >> Fmt<T>::M) & ((1u << Fmt<T>::E) - 1)) - Fmt<T>::BIAS;
}

// Mantissa bits an unpredictable value keeps: with x in [2^ex, 2^(ex+1)), dropping all but m
// mantissa bits errs by less than 2^(ex-m), which is at most 2^eexp <= eb once m >= ex - eexp.
// Zeros, subnormals, infinities and NaNs keep every bit.
template <typename T> int kept_mantissa_bits(T x, int eexp) {
  const int Ex = (int)((raw_bits<T>(x) >> Fmt<T>::M) & ((1u << Fmt<T>::E) - 1));
  if (Ex == 0 || Ex == (1 << Fmt<T>::E) - 1) return Fmt<T>::M;
  const int m = Ex - Fmt<T>::BIAS - eexp;
  return m < 0 ? 0 : (m > Fmt<T>::M ? Fmt<T>::M : m);
}

// The value an unpredictable point decompresses to: x with the dropped mantissa bits zero.
template <typename T> T truncate_unpredictable(T x, int eexp) {
  const int drop = Fmt<T>::M - kept_mantissa_bits<T>(x, eexp);
  typename Fmt<T>::U u = raw_bits<T>(x);
  if (drop > 0) u &= ~((((typename Fmt<T>::U)1) << drop) - 1);
  return from_raw<T>(u);
}

// ---------------------------------------------------------------- per-block compression
struct Ctx {
  Geom g;
  int predictor_mode = 0;
  bool abft = true;
  bool compact = false;
  uint32_t bins = 65536, R = 32768;
  const orc_flip* flips = nullptr;
  int nflips = 0;
};

template <typename T>
struct BlockResult {
  uint32_t ext[3];
  bool regression = false;
  T coef[4] = {0, 0, 0, 0};
  int32_t kq[4] = {0, 0, 0, 0};  // compact encoding: the stored coefficient integers
  std::vector<uint16_t> code;  // q_bin[] (Sec. 4.2.3): 0 = unpredictable, else q + R
  std::vector<T> vin;          // verified input values, the source of unpredictable values
  uint64_t sum_q = 0, isum_q = 0, sum_dc = 0;
  int input_status = 0;        // 0 clean, 1 corrected, 2 uncorrectable
  uint64_t dup_fixed = 0;
  uint64_t n_unpred = 0;
};

const orc_flip* find_flip(const Ctx& c, uint32_t site, uint64_t block, uint64_t index) {
  for (int n = 0; n < c.nflips; ++n)
    if (c.flips[n].site == site && c.flips[n].block == block && c.flips[n].index == index) return &c.flips[n];
  return nullptr;
}

// Prediction preparation for one block (Algorithm 1, Sec. 4.1.1): regression coefficients
// and the two error estimates, from the block's values as they are in the first pass.
struct Prep {
  float coef[4] = {0, 0, 0, 0};
  bool finite = false;
  float Ereg = 0.0f, Elor = 0.0f;
  int32_t kq[4] = {0, 0, 0, 0};  // compact encoding: the coefficients as multiples of their steps
};

template <typename T>
void load_block(const Geom& g, const T* field, uint64_t b, std::vector<T>* v, uint32_t ext[3]) {
  uint64_t org[3];
  block_box(g, b, org, ext);
  v->resize((uint64_t)ext[0] * ext[1] * ext[2]);
  uint64_t k = 0;
  for (uint32_t i = 0; i < ext[0]; ++i)
    for (uint32_t j = 0; j < ext[1]; ++j)
      for (uint32_t l = 0; l < ext[2]; ++l) (*v)[k++] = field[global_index(g, org, i, j, l)];
}

template <typename T>
Prep prepare_block(const Ctx& c, const T* field, uint64_t b) {
  std::vector<T> v;
  uint32_t e[3];
  load_block<T>(c.g, field, b, &v, e);
  Prep pr;
  pr.finite = regression_coefficients<T>(v.data(), e, c.g.ndim, pr.coef);
  if (pr.finite && c.predictor_mode == 0) selection_estimates<T>(v.data(), e, c.g.ndim, pr.coef, &pr.Ereg, &pr.Elor);
  return pr;
}

bool indicator_of(const Ctx& c, const Prep& pr, const uint32_t e[3], float ebf) {
  if (!pr.finite) return false;
  if (c.predictor_mode == 2) return true;
  if (c.predictor_mode == 1) return false;
  return select_regression(pr.Ereg, pr.Elor, sample_points(c.g.ndim, e), c.g.ndim, ebf);
}

// Compact encoding, once the bound is known: the coefficients become integers (a coefficient
// that cannot be one makes the block use Lorenzo), and the selection estimate of regression is
// taken with the coefficients the block would predict with, on the values of the first pass.
template <typename T>
void quantize_prep(const Ctx& c, const T* field, uint64_t b, T eb, Prep* pr) {
  if (!pr->finite) return;
  const CoefSteps qs = coef_steps(c.g, (double)eb);
  float cq[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int a = 0; a <= c.g.ndim; ++a) {
    if (!quantize_coef(pr->coef[a], qs.inv[a], &pr->kq[a])) {
      pr->finite = false;
      return;
    }
    cq[a] = (float)dequantize_coef<T>(pr->kq[a], qs.step[a]);
  }
  for (int a = 0; a < 4; ++a) pr->coef[a] = cq[a];
  if (c.predictor_mode == 0) {
    std::vector<T> v;
    uint32_t e[3];
    load_block<T>(c.g, field, b, &v, e);
    selection_estimates<T>(v.data(), e, c.g.ndim, pr->coef, &pr->Ereg, &pr->Elor);
  }
}

// Algorithm 1's prediction loop for one block: verify the input with sum_in/isum_in, pick f()
// from the indicator, then predict every point with duplicated prediction and
// reconstruction (f_dup, dec_dup) and take the block checksums (sum_q/isum_q, sum_dc).
template <typename T>
void compress_block(const Ctx& c, const T* field, uint64_t b, T eb, T inv2, uint64_t sum_in, uint64_t isum_in,
                    const Prep& pr, BlockResult<T>* out) {
  const Geom& g = c.g;
  std::vector<T>& v = out->vin;
  load_block<T>(g, field, b, &v, out->ext);
  const uint32_t* e = out->ext;
  const uint64_t P = (uint64_t)e[0] * e[1] * e[2];
  uint64_t k = 0;

  // memory-error detection and correction with sum_in / isum_in (Algorithm 1, Sec. 3.2)
  if (c.abft) {
    const int W = Bits<T>::kWords;
    std::vector<uint32_t> w(P * W);
    for (uint64_t p = 0; p < P; ++p) Bits<T>::words(v[p], &w[p * W]);
    out->input_status = locate_and_repair(w.data(), P * W, sum_in, isum_in, 0xffffffffull);
    if (out->input_status == 1)
      for (uint64_t p = 0; p < P; ++p) v[p] = Bits<T>::from_words(&w[p * W]);
  }

  const bool use_reg = indicator_of(c, pr, e, (float)eb);
  out->regression = use_reg;
  if (c.compact) {
    // the stored integers are what a memory error strikes; both sides dequantize them
    const CoefSteps qs = coef_steps(g, (double)eb);
    for (int a = 0; a < 4; ++a) out->kq[a] = pr.kq[a];
    for (int a = 0; a <= g.ndim; ++a) {
      const orc_flip* f = find_flip(c, SITE_COEF, b, (uint64_t)a);
      if (f) out->kq[a] = (int32_t)((uint32_t)out->kq[a] ^ (1u << (f->bit & 31)));
    }
    for (int a = 0; a < 4; ++a) out->coef[a] = a <= g.ndim ? dequantize_coef<T>(out->kq[a], qs.step[a]) : (T)0;
  } else {
    for (int a = 0; a < 4; ++a) out->coef[a] = (T)pr.coef[a];
    for (int a = 0; a <= g.ndim; ++a) {
      const orc_flip* f = find_flip(c, SITE_COEF, b, (uint64_t)a);
      if (f) out->coef[a] = Bits<T>::flip(out->coef[a], f->bit);
    }
  }
  const int eexp = bound_exponent<T>(eb);

  // the per-point loop
  const T Rh = (T)c.R - (T)0.5;
  std::vector<T> xrec(P);
  out->code.assign(P, 0);
  out->sum_q = out->isum_q = out->sum_dc = 0;
  out->n_unpred = 0;
  k = 0;
  for (uint32_t i = 0; i < e[0]; ++i)
    for (uint32_t j = 0; j < e[1]; ++j)
      for (uint32_t l = 0; l < e[2]; ++l, ++k) {
        uint32_t c3[3] = {i, j, l};
        auto predict = [&]() -> T {
          return use_reg ? regress<T>(out->coef, g.ndim, c3) : lorenzo<T>(xrec.data(), e, g.ndim, i, j, l);
        };
        // pred' <- f_dup(); a disagreement is settled by a third evaluation
        T pred = predict();
        if (c.abft) {
          const orc_flip* f = find_flip(c, SITE_PRED, b, k);
          if (f) pred = Bits<T>::flip(pred, f->bit);
          T pred2 = predict();
          if (!Bits<T>::same(pred, pred2)) {
            pred = predict();
            out->dup_fixed++;
          }
        }
        const T x = v[k];
        const T diff = x - pred;
        const T t = std::fabs(diff) * inv2;         // linear-scaling quantization
        uint16_t code = 0;
        T xr = x;
        if (t < Rh) {                               // bin within range (false for NaN)
          int32_t m = (int32_t)(t + (T)0.5);
          int32_t q = diff < (T)0 ? -m : m;
          auto decode = [&]() -> T { return pred + (T)(2 * q) * eb; };
          T xd = decode();                          // dcmp <- dec_dup(q, pred')
          if (c.abft) {
            const orc_flip* f = find_flip(c, SITE_RECON, b, k);
            if (f) xd = Bits<T>::flip(xd, f->bit);
            T xd2 = decode();
            if (!Bits<T>::same(xd, xd2)) {
              xd = decode();
              out->dup_fixed++;
            }
          }
          if (std::fabs(x - xd) <= eb) {            // double check vs machine epsilon (Sec. 4.1.2)
            code = (uint16_t)(q + (int32_t)c.R);
            xr = xd;
          }
        }
        if (code == 0) {                            // unpredictable: stored raw, or truncated
          out->n_unpred++;
          if (c.compact) xr = truncate_unpredictable<T>(x, eexp);
        }
        out->code[k] = code;
        xrec[k] = xr;
        out->sum_q += code;                         // sum_q, isum_q
        out->isum_q += (k + 1) * (uint64_t)code;
        uint32_t w[2] = {0, 0};
        Bits<T>::words(xr, w);
        for (int m = 0; m < Bits<T>::kWords; ++m) out->sum_dc += w[m];  // sum_dc
      }
}

// ---------------------------------------------------------------- Huffman (Algorithm 1)
// Code lengths for a histogram. Huffman's algorithm with a priority queue keyed by
// (weight, creation order): leaves are created in increasing (count, symbol) order, then
// internal nodes in the order they are formed. Lengths longer than kMaxLen are reduced
// with the JPEG adjustment (ITU-T T.81 Annex K.3). The final lengths are handed out
// longest-first to the leaves in increasing (count, symbol) order.
void huffman_lengths(const uint64_t* hist, uint32_t nsym, uint8_t* len) {
  std::memset(len, 0, nsym);
  std::vector<uint32_t> leaves;
  for (uint32_t s = 0; s < nsym; ++s)
    if (hist[s]) leaves.push_back(s);
  const uint32_t n = (uint32_t)leaves.size();
  if (n == 0) return;
  std::stable_sort(leaves.begin(), leaves.end(),
                   [&](uint32_t a, uint32_t b) { return hist[a] != hist[b] ? hist[a] < hist[b] : a < b; });
  if (n == 1) {
    len[leaves[0]] = 1;
    return;
  }
  // nodes 0..n-1 are leaves (in sorted order), n..2n-2 internal
  std::vector<uint64_t> weight(2 * n - 1);
  std::vector<uint32_t> parent(2 * n - 1, 0);
  typedef std::pair<uint64_t, uint32_t> Key;  // (weight, node id == creation order)
  std::priority_queue<Key, std::vector<Key>, std::greater<Key>> pq;
  for (uint32_t p = 0; p < n; ++p) {
    weight[p] = hist[leaves[p]];
    pq.push(Key(weight[p], p));
  }
  uint32_t next = n;
  while (pq.size() > 1) {
    Key a = pq.top(); pq.pop();
    Key b = pq.top(); pq.pop();
    weight[next] = a.first + b.first;
    parent[a.second] = next;
    parent[b.second] = next;
    pq.push(Key(weight[next], next));
    ++next;
  }
  // depth of every node: the root is the last node formed
  std::vector<uint32_t> depth(2 * n - 1, 0);
  for (int64_t v = (int64_t)(2 * n - 3); v >= 0; --v) depth[v] = depth[parent[v]] + 1;
  std::vector<uint64_t> count(64, 0);
  uint32_t maxlen = 0;
  for (uint32_t p = 0; p < n; ++p) {
    count[depth[p]]++;
    maxlen = std::max(maxlen, depth[p]);
  }
  // JPEG Annex K.3 length limiting: move pairs from the deepest level up.
  for (uint32_t l = maxlen; l > kMaxLen; --l) {
    while (count[l] > 0) {
      uint32_t j = l - 2;
      while (count[j] == 0) --j;
      count[l] -= 2;
      count[l - 1] += 1;
      count[j + 1] += 2;
      count[j] -= 1;
    }
  }
  // longest lengths to the rarest leaves
  uint32_t p = 0;
  for (uint32_t l = std::min(maxlen, kMaxLen); l >= 1 && p < n; --l)
    for (uint64_t c = 0; c < count[l]; ++c) len[leaves[p++]] = (uint8_t)l;
}

// Canonical code assignment: symbols ordered by (length, symbol) receive consecutive codes.
struct Canon {
  uint32_t bl_count[kMaxLen + 1] = {0};
  uint32_t first_code[kMaxLen + 2] = {0};
  uint32_t first_index[kMaxLen + 2] = {0};
  std::vector<uint16_t> symbols;  // canonical order
};

void canon_from_counts(Canon* c) {
  uint32_t code = 0, idx = 0;
  for (uint32_t l = 1; l <= kMaxLen; ++l) {
    code = (code + (l >= 2 ? c->bl_count[l - 1] : 0)) << 1;
    c->first_code[l] = code;
    c->first_index[l] = idx;
    idx += c->bl_count[l];
  }
}

void canon_from_lengths(const uint8_t* len, uint32_t nsym, Canon* c, std::vector<uint32_t>* code_of) {
  std::memset(c->bl_count, 0, sizeof(c->bl_count));
  c->symbols.clear();
  for (uint32_t l = 1; l <= kMaxLen; ++l)
    for (uint32_t s = 0; s < nsym; ++s)
      if (len[s] == l) {
        c->symbols.push_back((uint16_t)s);
        c->bl_count[l]++;
      }
  canon_from_counts(c);
  code_of->assign(nsym, 0);
  for (uint32_t l = 1; l <= kMaxLen; ++l)
    for (uint32_t r = 0; r < c->bl_count[l]; ++r) (*code_of)[c->symbols[c->first_index[l] + r]] = c->first_code[l] + r;
}

struct BitWriter {
  std::vector<uint8_t> bytes;
  uint64_t nbits = 0;
  void put(uint64_t code, uint32_t len) {  // the low len bits of code, MSB-first
    for (int s = (int)len - 1; s >= 0; --s) {
      if (nbits % 8 == 0) bytes.push_back(0);
      if ((code >> s) & 1u) bytes.back() |= (uint8_t)(0x80u >> (nbits % 8));
      ++nbits;
    }
  }
};

// Compact encoding: a coefficient integer as its zigzag value z (0, -1, 1, -2, ... -> 0, 1, 2,
// 3, ...), written as the bit length n of z in 6 bits, then the n - 1 bits of z below its
// leading one.
void put_coef_int(BitWriter* bw, int32_t k) {
  const uint32_t z = ((uint32_t)k << 1) ^ (k < 0 ? 0xffffffffu : 0u);
  uint32_t n = 0;
  while (n < 32 && (z >> n) != 0) ++n;
  bw->put(n, 6);
  if (n > 1) bw->put(z & ((1u << (n - 1)) - 1u), n - 1);
}

// Compact encoding: an unpredictable value as its sign, exponent and kept mantissa bits.
template <typename T>
void put_unpredictable(BitWriter* bw, T x, int eexp) {
  const int m = kept_mantissa_bits<T>(x, eexp);
  bw->put((uint64_t)(raw_bits<T>(x) >> (Fmt<T>::M - m)), (uint32_t)(1 + Fmt<T>::E + m));
}

// ---------------------------------------------------------------- stream layout
uint64_t align16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

struct Layout {
  uint64_t table, groups, sizes, ucounts, bitmap, sumdc, coef, unpred, payload;
};

// The compact encoding keeps coefficients and unpredictable values in the payload, so its
// coefficient and unpredictable sections are empty.
Layout make_layout(const Geom& g, bool abft, bool compact, uint64_t n_live, uint64_t n_reg, uint64_t n_unpred) {
  const uint64_t s = g.dtype ? 8 : 4;
  const uint64_t ngroups = (g.nb + kGroup - 1) / kGroup;
  Layout L;
  L.table = kHeader;
  L.groups = align16(L.table + 4 * (kMaxLen + 1) + 2 * n_live);
  L.sizes = align16(L.groups + 24 * ngroups);
  L.ucounts = align16(L.sizes + 2 * g.nb);
  L.bitmap = align16(L.ucounts + 2 * g.nb);
  L.sumdc = align16(L.bitmap + 4 * ((g.nb + 31) / 32));
  L.coef = align16(L.sumdc + (abft ? 8 * g.nb : 0));
  L.unpred = align16(L.coef + (compact ? 0 : s * (uint64_t)(g.ndim + 1) * n_reg));
  L.payload = align16(L.unpred + (compact ? 0 : s * n_unpred));
  return L;
}

template <typename V> void put(uint8_t* o, uint64_t off, V v) { std::memcpy(o + off, &v, sizeof(V)); }
template <typename V> V get(const uint8_t* o, uint64_t off) { V v; std::memcpy(&v, o + off, sizeof(V)); return v; }

// ---------------------------------------------------------------- Alg. 1
template <typename T>
int compress_impl(const T* field_in, const orc_params* p, const orc_flip* flips, int nflips, uint8_t* out,
                  uint64_t cap, uint64_t* out_bytes, orc_report* rep) {
  Ctx c;
  if (!make_geom(p, &c.g)) return EINVAL_;
  const Geom& g = c.g;
  if (!(p->eb > 0.0) || !std::isfinite(p->eb) || p->eb_mode > 1) return EINVAL_;
  if (p->quant_bins < 2 || p->quant_bins > 65536 || (p->quant_bins & 1)) return EINVAL_;
  if (p->predictor > 2 || p->encoding > 3) return EINVAL_;
  c.compact = (p->encoding & 1) != 0;
  c.bins = p->quant_bins;
  c.R = p->quant_bins / 2;
  c.abft = p->abft != 0;
  c.predictor_mode = (int)p->predictor;
  c.flips = flips;
  c.nflips = nflips;

  // Algorithm 1's first loops: per block input checksums,
  // regression coefficients and selection estimates; the value range for the bound.
  std::vector<uint64_t> sum_in(g.nb, 0), isum_in(g.nb, 0);
  std::vector<Prep> prep(g.nb);
  for (uint64_t b = 0; b < g.nb; ++b) {
    prep[b] = prepare_block<T>(c, field_in, b);
    if (c.abft) {
      std::vector<T> v;
      uint32_t e[3];
      load_block<T>(g, field_in, b, &v, e);
      const int W = Bits<T>::kWords;
      std::vector<uint32_t> w(v.size() * W);
      for (uint64_t p = 0; p < v.size(); ++p) Bits<T>::words(v[p], &w[p * W]);
      checksum_words(w.data(), w.size(), &sum_in[b], &isum_in[b]);
    }
  }
  // Error bound: absolute, or value-range relative over the finite values (Fig. 2 caption).
  double ebd = p->eb;
  if (p->eb_mode == 1) {
    bool any = false;
    T mn = 0, mx = 0;
    for (uint64_t n = 0; n < g.N; ++n) {
      T x = field_in[n];
      if (!std::isfinite(x)) continue;
      if (!any) { mn = mx = x; any = true; }
      if (x < mn) mn = x;
      if (x > mx) mx = x;
    }
    if (any && mx > mn) ebd = p->eb * ((double)mx - (double)mn);
  }
  const T eb = (T)ebd;
  if (!(eb > (T)0) || !std::isfinite(eb) || !std::isnormal(eb)) return EINVAL_;
  const T inv2 = (T)(1.0 / (2.0 * (double)eb));
  if (c.compact)
    for (uint64_t b = 0; b < g.nb; ++b) quantize_prep<T>(c, field_in, b, eb, &prep[b]);

  std::vector<T> field(field_in, field_in + g.N);  // working copy that soft errors may strike
  // memory errors in the input strike here, after its checksums (Sec. 6.1.2, mode A)
  for (int n = 0; n < nflips; ++n)
    if (flips[n].site == SITE_INPUT) {
      uint64_t word = flips[n].index;
      uint64_t pt = word / Bits<T>::kWords;
      if (pt >= g.N) continue;
      uint32_t w[2];
      Bits<T>::words(field[pt], w);
      w[word % Bits<T>::kWords] ^= (1u << (flips[n].bit & 31));
      field[pt] = Bits<T>::from_words(w);
    }

  // Algorithm 1's prediction loop, one block at a time; the histogram is taken as codes are made.
  std::vector<BlockResult<T>> blk(g.nb);
  std::vector<uint64_t> hist(c.bins, 0);
  orc_report r;
  std::memset(&r, 0, sizeof(r));
  r.blocks = g.nb;
  r.eb_abs = (double)eb;
  for (uint64_t b = 0; b < g.nb; ++b) {
    compress_block<T>(c, field.data(), b, eb, inv2, sum_in[b], isum_in[b], prep[b], &blk[b]);
    for (uint16_t q : blk[b].code) hist[q]++;
    if (blk[b].input_status == 1) r.input_corrected++;
    if (blk[b].input_status == 2) r.uncorrectable_blocks++;
    r.dup_mismatch_corrected += blk[b].dup_fixed;
  }
  // memory errors in the bin array strike here, after sum_q / isum_q (Sec. 4.2.3)
  for (int n = 0; n < nflips; ++n)
    if (flips[n].site == SITE_CODE && flips[n].block < g.nb && flips[n].index < blk[flips[n].block].code.size())
      blk[flips[n].block].code[flips[n].index] ^= (uint16_t)(1u << (flips[n].bit & 15));

  // one Huffman code for the whole bin array (Algorithm 1)
  std::vector<uint8_t> len(c.bins);
  huffman_lengths(hist.data(), c.bins, len.data());
  Canon canon;
  std::vector<uint32_t> code_of;
  canon_from_lengths(len.data(), c.bins, &canon, &code_of);

  // verify each block's codes with sum_q/isum_q, then encode the block on its own (Algorithm 1)
  std::vector<std::vector<uint8_t>> payload(g.nb);
  std::vector<uint32_t> ucount(g.nb, 0);
  uint64_t n_unpred = 0, n_reg = 0, payload_bytes = 0;
  for (uint64_t b = 0; b < g.nb; ++b) {
    BlockResult<T>& B = blk[b];
    const uint64_t P = B.code.size();
    if (c.abft) {
      std::vector<uint32_t> w(B.code.begin(), B.code.end());
      int st = locate_and_repair(w.data(), P, B.sum_q, B.isum_q, (uint64_t)c.bins - 1);
      if (st == 1) {
        r.codes_corrected++;
        for (uint64_t k = 0; k < P; ++k) B.code[k] = (uint16_t)w[k];
      } else if (st == 2) {
        r.uncorrectable_blocks++;
      }
    }
    BitWriter bw;
    if (c.compact && B.regression)
      for (int a = 0; a <= g.ndim; ++a) put_coef_int(&bw, B.kq[a]);
    const int eexp = bound_exponent<T>(eb);
    for (uint64_t k = 0; k < P; ++k) {
      uint16_t q = B.code[k];
      if (q == 0) ucount[b]++;
      bw.put(code_of[q], len[q]);
      if (q == 0 && c.compact) put_unpredictable<T>(&bw, B.vin[k], eexp);
    }
    payload[b] = bw.bytes;
    payload_bytes += bw.bytes.size();
    n_unpred += ucount[b];
    if (B.regression) n_reg++;
  }
  r.regression_blocks = n_reg;
  r.unpredictable_points = n_unpred;

  // write the stream (Algorithm 1's output step, without the Zstd stage)
  const uint64_t s = sizeof(T);
  const uint64_t n_live = canon.symbols.size();
  Layout L = make_layout(g, c.abft, c.compact, n_live, n_reg, n_unpred);
  const uint64_t total = L.payload + payload_bytes;
  if (total > cap) return ECAPACITY;
  std::memset(out, 0, total);
  std::memcpy(out, "SDSZ", 4);
  put<uint16_t>(out, 4, 1);
  put<uint8_t>(out, 6, (uint8_t)g.dtype);
  put<uint8_t>(out, 7, (uint8_t)g.ndim);
  for (int a = 0; a < 3; ++a) put<uint64_t>(out, 8 + 8 * a, a < g.ndim ? p->dims[a] : 0);
  for (int a = 0; a < 3; ++a) put<uint32_t>(out, 32 + 4 * a, a < g.ndim ? p->block[a] : 0);
  put<uint32_t>(out, 44, c.bins);
  put<uint8_t>(out, 48, (uint8_t)c.abft);
  put<uint8_t>(out, 49, (uint8_t)p->predictor);
  put<uint8_t>(out, 50, (uint8_t)p->eb_mode);
  put<uint8_t>(out, 51, (uint8_t)(p->encoding & 1));  // the lossless stage sets bit 1 itself
  put<uint32_t>(out, 52, (uint32_t)n_live);
  put<double>(out, 56, (double)eb);
  put<double>(out, 64, p->eb);
  put<uint64_t>(out, 72, g.nb);
  put<uint64_t>(out, 80, n_reg);
  put<uint64_t>(out, 88, n_unpred);
  put<uint64_t>(out, 96, payload_bytes);
  put<uint64_t>(out, 104, total);
  put<uint32_t>(out, 112, r.uncorrectable_blocks ? 1u : 0u);
  for (uint32_t l = 0; l <= kMaxLen; ++l) put<uint32_t>(out, L.table + 4 * l, canon.bl_count[l]);
  for (uint64_t n = 0; n < n_live; ++n) put<uint16_t>(out, L.table + 4 * (kMaxLen + 1) + 2 * n, canon.symbols[n]);
  uint64_t pay = 0, un = 0, rg = 0;
  for (uint64_t b = 0; b < g.nb; ++b) {
    if (b % kGroup == 0) {
      uint64_t gi = b / kGroup;
      put<uint64_t>(out, L.groups + 24 * gi, pay);
      put<uint64_t>(out, L.groups + 24 * gi + 8, un);
      put<uint64_t>(out, L.groups + 24 * gi + 16, rg);
    }
    const BlockResult<T>& B = blk[b];
    put<uint16_t>(out, L.sizes + 2 * b, (uint16_t)payload[b].size());
    put<uint16_t>(out, L.ucounts + 2 * b, (uint16_t)ucount[b]);
    if (B.regression) {
      uint32_t word = get<uint32_t>(out, L.bitmap + 4 * (b / 32));
      put<uint32_t>(out, L.bitmap + 4 * (b / 32), word | (1u << (b % 32)));
      if (!c.compact)
        for (int a = 0; a <= g.ndim; ++a) put<T>(out, L.coef + s * ((g.ndim + 1) * rg + a), B.coef[a]);
      rg++;
    }
    if (c.abft) put<uint64_t>(out, L.sumdc + 8 * b, B.sum_dc);
    if (c.compact) un += ucount[b];
    else
      for (uint64_t k = 0; k < B.code.size(); ++k)
        if (B.code[k] == 0) put<T>(out, L.unpred + s * un++, B.vin[k]);
    if (!payload[b].empty()) std::memcpy(out + L.payload + pay, payload[b].data(), payload[b].size());
    pay += payload[b].size();
  }
  r.compressed_bytes = total;
  if (out_bytes) *out_bytes = total;
  if (rep) *rep = r;
  return OK;
}

// ---------------------------------------------------------------- lossless stage
// Algorithm 1 ends by compressing the encoded bin array (and sum_dc) losslessly, Algorithm 2
// starts by undoing that; the paper uses Zstd. Here: an order-0 range asymmetric numeral system
// (rANS) coder over the bytes from the sum_dc section to the end of the stream. Everything
// before it (header, code table and the random-access tables) stays as it is.
//   * symbol frequencies: the byte counts scaled to 4096 (12 bits); a byte that occurs gets at
//     least 1; the sum is then brought to 4096 one step at a time, taking from the largest
//     frequency above 1 (ties: smaller byte) or giving to the most frequent byte (ties:
//     smaller byte);
//   * the bytes are cut into chunks of 16384; in a chunk, byte i belongs to state i mod 32;
//   * state x in [2^16, 2^32); coding s (frequency f, cumulative c) first renormalises,
//     emitting the low 16 bits while x >= 2^20 f, then x <- (x / f) 2^12 + x mod f + c;
//     decoding is the inverse: slot = x mod 2^12, s = the byte whose range holds slot,
//     x <- f (x / 2^12) + slot - c, then x <- x 2^16 + the next word while x < 2^16;
//   * the coder runs over the chunk from its last byte to its first; the 16-bit words are
//     stored in the order the decoder takes them (byte order, states in increasing index at
//     each byte group), after the 32 final states;
//   * section layout at the sum_dc offset: 256 frequencies (u16), the end offset of each
//     chunk (u32, relative to the first chunk, whose start is 16-byte aligned), then the
//     chunks, each padded to 4 bytes. Header: byte 51 bit 1 set, the total at 104 is the
//     stream's, the total without the stage at 120.
constexpr uint32_t kLLChunk = 16384, kLLScale = 12, kLLM = 1u << kLLScale, kLLWays = 32;
constexpr uint64_t kRansLow = 1ull << 16;

void ll_frequencies(const uint64_t cnt[256], uint16_t f[256]) {
  uint64_t total = 0;
  for (int b = 0; b < 256; ++b) total += cnt[b];
  std::memset(f, 0, 256 * sizeof(uint16_t));
  if (!total) return;
  int64_t sum = 0;
  uint32_t fw[256];
  for (int b = 0; b < 256; ++b) {
    fw[b] = 0;
    if (cnt[b]) {
      const uint64_t v = cnt[b] * kLLM / total;
      fw[b] = v < 1 ? 1u : (uint32_t)v;
    }
    sum += fw[b];
  }
  while (sum > (int64_t)kLLM) {
    int best = -1;
    for (int b = 0; b < 256; ++b)
      if (fw[b] > 1 && (best < 0 || fw[b] > fw[best])) best = b;
    --fw[best];
    --sum;
  }
  while (sum < (int64_t)kLLM) {
    int best = 0;
    for (int b = 1; b < 256; ++b)
      if (cnt[b] > cnt[best]) best = b;
    ++fw[best];
    ++sum;
  }
  for (int b = 0; b < 256; ++b) f[b] = (uint16_t)fw[b];
}

void ll_cumulative(const uint16_t f[256], uint32_t c[257]) {
  c[0] = 0;
  for (int b = 0; b < 256; ++b) c[b + 1] = c[b] + f[b];
}

// One chunk: 32 final states (u32) then the words in decoding order, padded to 4 bytes.
void ll_encode_chunk(const uint8_t* in, uint32_t n, const uint16_t f[256], const uint32_t c[257],
                     std::vector<uint8_t>* out) {
  uint64_t x[kLLWays];
  for (uint32_t j = 0; j < kLLWays; ++j) x[j] = kRansLow;
  std::vector<uint16_t> pushed;  // in the order the coder emits them
  const uint32_t T = (n + kLLWays - 1) / kLLWays;
  for (uint32_t t = T; t-- > 0;)
    for (uint32_t j = kLLWays; j-- > 0;) {
      const uint32_t i = t * kLLWays + j;
      if (i >= n) continue;
      const uint32_t s = in[i], fs = f[s];
      const uint64_t xmax = (uint64_t)((kRansLow >> kLLScale) << 16) * fs;
      if (x[j] >= xmax) {
        pushed.push_back((uint16_t)(x[j] & 0xffff));
        x[j] >>= 16;
      }
      x[j] = ((x[j] / fs) << kLLScale) + (x[j] % fs) + c[s];
    }
  const size_t at = out->size();
  out->resize(at + 4 * kLLWays + 2 * pushed.size());
  for (uint32_t j = 0; j < kLLWays; ++j) put<uint32_t>(out->data(), at + 4 * j, (uint32_t)x[j]);
  for (size_t q = 0; q < pushed.size(); ++q)
    put<uint16_t>(out->data(), at + 4 * kLLWays + 2 * q, pushed[pushed.size() - 1 - q]);
  if (out->size() & 3) out->resize(out->size() + 2, 0);
}

// Decode n bytes of one chunk of `len` bytes; words past the chunk read as 0.
void ll_decode_chunk(const uint8_t* in, uint64_t len, uint32_t n, const uint16_t f[256], const uint32_t c[257],
                     const uint8_t* sym, uint8_t* out) {
  uint64_t x[kLLWays];
  for (uint32_t j = 0; j < kLLWays; ++j) x[j] = 4 * (j + 1) <= len ? get<uint32_t>(in, 4 * j) : 0;
  const uint64_t nw = len > 4 * kLLWays ? (len - 4 * kLLWays) / 2 : 0;
  uint64_t p = 0;
  const uint32_t T = (n + kLLWays - 1) / kLLWays;
  for (uint32_t t = 0; t < T; ++t)
    for (uint32_t j = 0; j < kLLWays; ++j) {
      const uint32_t i = t * kLLWays + j;
      if (i >= n) continue;
      const uint32_t slot = (uint32_t)(x[j] & (kLLM - 1));
      const uint32_t s = sym[slot];
      out[i] = (uint8_t)s;
      x[j] = (uint64_t)f[s] * (x[j] >> kLLScale) + slot - c[s];
      if (x[j] < kRansLow) {
        const uint64_t w = p < nw ? get<uint16_t>(in, 4 * kLLWays + 2 * p) : 0;
        ++p;
        x[j] = ((x[j] << 16) | w) & 0xffffffffull;
      }
    }
}

// The lossless stage over a finished stream R whose coded region starts at `from`.
void ll_pack(const uint8_t* R, uint64_t nR, uint64_t from, uint8_t encoding, std::vector<uint8_t>* S) {
  uint64_t cnt[256] = {0};
  for (uint64_t q = from; q < nR; ++q) cnt[R[q]]++;
  uint16_t f[256];
  uint32_t c[257];
  ll_frequencies(cnt, f);
  ll_cumulative(f, c);
  const uint64_t n = nR - from, nchunks = (n + kLLChunk - 1) / kLLChunk;
  const uint64_t data = align16(from + 512 + 4 * nchunks);
  std::vector<uint8_t> chunks;
  std::vector<uint32_t> ends(nchunks);
  for (uint64_t k = 0; k < nchunks; ++k) {
    const uint32_t len = (uint32_t)std::min<uint64_t>(kLLChunk, n - k * kLLChunk);
    ll_encode_chunk(R + from + k * kLLChunk, len, f, c, &chunks);
    ends[k] = (uint32_t)chunks.size();
  }
  S->assign(data + chunks.size(), 0);
  std::memcpy(S->data(), R, from);
  put<uint8_t>(S->data(), 51, (uint8_t)(encoding | 2));
  put<uint64_t>(S->data(), 104, (uint64_t)S->size());
  put<uint64_t>(S->data(), 120, nR);
  for (int b = 0; b < 256; ++b) put<uint16_t>(S->data(), from + 2 * b, f[b]);
  for (uint64_t k = 0; k < nchunks; ++k) put<uint32_t>(S->data(), from + 512 + 4 * k, ends[k]);
  if (!chunks.empty()) std::memcpy(S->data() + data, chunks.data(), chunks.size());
}

// Undo the lossless stage: R is the stream without it. False when the section is malformed.
bool ll_unpack(const uint8_t* S, uint64_t nS, uint64_t from, uint64_t nR, std::vector<uint8_t>* R) {
  if (nR < from || from + 512 > nS) return false;
  const uint64_t n = nR - from, nchunks = (n + kLLChunk - 1) / kLLChunk;
  const uint64_t data = align16(from + 512 + 4 * nchunks);
  if (data > nS) return false;
  uint16_t f[256];
  for (int b = 0; b < 256; ++b) f[b] = get<uint16_t>(S, from + 2 * b);
  uint32_t c[257];
  ll_cumulative(f, c);
  if (n && c[256] != kLLM) return false;
  std::vector<uint8_t> sym(kLLM, 0);
  for (int b = 0; b < 256; ++b)
    for (uint32_t q = c[b]; q < c[b + 1]; ++q) sym[q] = (uint8_t)b;
  R->assign(nR, 0);
  std::memcpy(R->data(), S, from);
  put<uint8_t>(R->data(), 51, (uint8_t)(S[51] & 1));
  put<uint64_t>(R->data(), 104, nR);
  put<uint64_t>(R->data(), 120, 0);
  uint64_t start = 0;
  for (uint64_t k = 0; k < nchunks; ++k) {
    const uint64_t end = get<uint32_t>(S, from + 512 + 4 * k);
    if (end < start || (end & 3) || data + end > nS) return false;
    const uint32_t len = (uint32_t)std::min<uint64_t>(kLLChunk, n - k * kLLChunk);
    ll_decode_chunk(S + data + start, end - start, len, f, c, sym.data(), R->data() + from + k * kLLChunk);
    start = end;
  }
  return true;
}

// ---------------------------------------------------------------- Alg. 2
struct Parsed {
  Geom g;
  orc_params p;
  uint32_t bins, R, n_live;
  bool abft, compact, lossless;
  double eb;
  uint64_t n_reg, n_unpred, payload_bytes, total;
  uint64_t raw_total;  // size of the stream without the lossless stage (= total without it)
  Layout L;
  Canon canon;
};

int parse(const uint8_t* s, uint64_t n, Parsed* P) {
  if (n < kHeader || std::memcmp(s, "SDSZ", 4) != 0 || get<uint16_t>(s, 4) != 1) return EFORMAT;
  std::memset(&P->p, 0, sizeof(P->p));
  P->p.dtype = get<uint8_t>(s, 6);
  P->p.ndim = get<uint8_t>(s, 7);
  if (P->p.ndim < 1 || P->p.ndim > 3 || P->p.dtype > 1) return EFORMAT;
  for (int a = 0; a < 3; ++a) P->p.dims[a] = get<uint64_t>(s, 8 + 8 * a);
  for (int a = 0; a < 3; ++a) P->p.block[a] = get<uint32_t>(s, 32 + 4 * a);
  P->bins = get<uint32_t>(s, 44);
  if (P->bins < 2 || P->bins > 65536 || (P->bins & 1)) return EFORMAT;
  P->R = P->bins / 2;
  P->p.quant_bins = P->bins;
  P->abft = get<uint8_t>(s, 48) != 0;
  P->p.abft = P->abft;
  P->p.predictor = get<uint8_t>(s, 49);
  P->p.eb_mode = get<uint8_t>(s, 50);
  P->p.encoding = get<uint8_t>(s, 51);
  if (P->p.encoding > 3) return EFORMAT;
  P->compact = (P->p.encoding & 1) != 0;
  P->lossless = (P->p.encoding & 2) != 0;
  P->n_live = get<uint32_t>(s, 52);
  P->eb = get<double>(s, 56);
  P->p.eb = get<double>(s, 64);
  if (!make_geom(&P->p, &P->g)) return EFORMAT;
  if (get<uint64_t>(s, 72) != P->g.nb) return EFORMAT;
  P->n_reg = get<uint64_t>(s, 80);
  P->n_unpred = get<uint64_t>(s, 88);
  P->payload_bytes = get<uint64_t>(s, 96);
  P->total = get<uint64_t>(s, 104);
  if (P->n_live > P->bins || P->n_reg > P->g.nb || P->n_unpred > P->g.N) return EFORMAT;
  P->L = make_layout(P->g, P->abft, P->compact, P->n_live, P->n_reg, P->n_unpred);
  P->raw_total = P->lossless ? get<uint64_t>(s, 120) : P->total;
  if (P->raw_total != P->L.payload + P->payload_bytes || P->total > n) return EFORMAT;
  uint64_t kraft = 0, cnt = 0;
  for (uint32_t l = 0; l <= kMaxLen; ++l) {
    P->canon.bl_count[l] = get<uint32_t>(s, P->L.table + 4 * l);
    if (l == 0 && P->canon.bl_count[0] != 0) return EFORMAT;
    kraft += (uint64_t)P->canon.bl_count[l] << (kMaxLen - l);
    cnt += P->canon.bl_count[l];
  }
  if (cnt != P->n_live || kraft > (1ull << kMaxLen)) return EFORMAT;
  P->canon.symbols.resize(P->n_live);
  for (uint64_t k = 0; k < P->n_live; ++k) {
    P->canon.symbols[k] = get<uint16_t>(s, P->L.table + 4 * (kMaxLen + 1) + 2 * k);
    if (P->canon.symbols[k] >= P->bins) return EFORMAT;
  }
  canon_from_counts(&P->canon);
  return OK;
}

// Decode one symbol, reading bits MSB-first from [bit, end). Returns -1 on an invalid code
// or when the block's bytes run out.
int decode_symbol(const uint8_t* pay, uint64_t* bit, uint64_t end, const Canon& c) {
  uint32_t code = 0;
  for (uint32_t l = 1; l <= kMaxLen; ++l) {
    if (*bit >= end) return -1;
    uint32_t b = (pay[*bit / 8] >> (7 - (*bit % 8))) & 1u;
    ++*bit;
    code = (code << 1) | b;
    if (c.bl_count[l] && code >= c.first_code[l] && code - c.first_code[l] < c.bl_count[l])
      return c.symbols[c.first_index[l] + (code - c.first_code[l])];
  }
  return -1;
}

// n raw bits (n <= 32) MSB-first from [bit, end); false when the block's bytes run out.
bool read_bits(const uint8_t* pay, uint64_t* bit, uint64_t end, uint32_t n, uint32_t* v) {
  uint32_t x = 0;
  for (uint32_t t = 0; t < n; ++t) {
    if (*bit >= end) return false;
    x = (x << 1) | ((pay[*bit / 8] >> (7 - (*bit % 8))) & 1u);
    ++*bit;
  }
  *v = x;
  return true;
}

// Compact encoding: one length-prefixed zigzag coefficient integer.
bool read_coef_int(const uint8_t* pay, uint64_t* bit, uint64_t end, int32_t* k) {
  uint32_t n, low = 0;
  if (!read_bits(pay, bit, end, 6, &n) || n > 32) return false;
  if (n > 1 && !read_bits(pay, bit, end, n - 1, &low)) return false;
  const uint32_t z = n == 0 ? 0u : ((n > 1 ? (1u << (n - 1)) : 1u) | low);
  *k = (int32_t)((z >> 1) ^ (0u - (z & 1u)));
  return true;
}

// Compact encoding: one truncated unpredictable value (sign, exponent, kept mantissa bits).
template <typename T>
bool read_unpredictable(const uint8_t* pay, uint64_t* bit, uint64_t end, int eexp, T* x) {
  typedef typename Fmt<T>::U U;
  uint32_t se;
  if (!read_bits(pay, bit, end, 1 + Fmt<T>::E, &se)) return false;
  const int Ex = (int)(se & ((1u << Fmt<T>::E) - 1));
  int m = Fmt<T>::M;
  if (Ex != 0 && Ex != (1 << Fmt<T>::E) - 1) {
    m = Ex - Fmt<T>::BIAS - eexp;
    m = m < 0 ? 0 : (m > Fmt<T>::M ? Fmt<T>::M : m);
  }
  U mant = 0;
  for (int got = 0; got < m;) {
    const uint32_t n = (uint32_t)std::min(32, m - got);
    uint32_t v;
    if (!read_bits(pay, bit, end, n, &v)) return false;
    mant = (mant << n) | v;
    got += (int)n;
  }
  const U u = ((U)se << Fmt<T>::M) | (mant << (Fmt<T>::M - m));
  *x = from_raw<T>(u);
  return true;
}

// One block of Algorithm 2's decompression loop: Huffman decode, then Lorenzo or regression.
// Returns false on a malformed block.
template <typename T>
bool decompress_block(const Parsed& P, const uint8_t* s, uint64_t b, uint64_t pay_off, uint64_t un_off,
                      int64_t reg_idx, const orc_flip* flips, int nflips, bool inject, T* out_block,
                      uint64_t* sumdc) {
  const Geom& g = P.g;
  uint64_t org[3];
  uint32_t e[3];
  block_box(g, b, org, e);
  const uint64_t Pn = (uint64_t)e[0] * e[1] * e[2];
  const uint64_t size = get<uint16_t>(s, P.L.sizes + 2 * b);
  const uint64_t ucnt = get<uint16_t>(s, P.L.ucounts + 2 * b);
  const T eb = (T)P.eb;
  const uint64_t sz = sizeof(T);
  T coef[4] = {0, 0, 0, 0};
  const uint8_t* pay = s + P.L.payload + pay_off;
  uint64_t bit = 0;
  const uint64_t end = 8 * size;
  uint64_t used = 0, k = 0;
  bool ok = true;
  const int eexp = bound_exponent<T>(eb);
  if (reg_idx >= 0 && P.compact) {
    const CoefSteps qs = coef_steps(g, (double)eb);
    for (int a = 0; a <= g.ndim && ok; ++a) {
      int32_t kq;
      ok = read_coef_int(pay, &bit, end, &kq);
      if (ok) coef[a] = dequantize_coef<T>(kq, qs.step[a]);
    }
  } else if (reg_idx >= 0) {
    for (int a = 0; a <= g.ndim; ++a) coef[a] = get<T>(s, P.L.coef + sz * ((g.ndim + 1) * (uint64_t)reg_idx + a));
  }
  uint64_t sum = 0;
  for (uint32_t i = 0; i < e[0]; ++i)
    for (uint32_t j = 0; j < e[1]; ++j)
      for (uint32_t l = 0; l < e[2]; ++l, ++k) {
        int q = ok ? decode_symbol(pay, &bit, end, P.canon) : -1;
        T xr = 0;
        if (q < 0) {
          ok = false;
        } else if (q == 0) {
          if (used >= ucnt) ok = false;
          else if (P.compact) ok = read_unpredictable<T>(pay, &bit, end, eexp, &xr);
          else xr = get<T>(s, P.L.unpred + sz * (un_off + used));
          if (!ok) xr = 0;
          ++used;
        } else {
          uint32_t c3[3] = {i, j, l};
          T pred = reg_idx >= 0 ? regress<T>(coef, g.ndim, c3) : lorenzo<T>(out_block, e, g.ndim, i, j, l);
          xr = pred + (T)(2 * (q - (int)P.R)) * eb;
        }
        if (inject)
          for (int n = 0; n < nflips; ++n)
            if (flips[n].site == SITE_DECOMP && flips[n].block == b && flips[n].index == k) xr = Bits<T>::flip(xr, flips[n].bit);
        out_block[k] = xr;
        uint32_t w[2] = {0, 0};
        Bits<T>::words(xr, w);
        for (int m = 0; m < Bits<T>::kWords; ++m) sum += w[m];
      }
  if (used != ucnt) ok = false;
  (void)Pn;
  *sumdc = sum;
  return ok;
}

template <typename T>
int decompress_impl(const uint8_t* s, uint64_t n, T* field, uint8_t* status, const orc_flip* flips, int nflips,
                    orc_report* rep) {
  Parsed P;
  int rc = parse(s, n, &P);
  if (rc) return rc;
  if (P.lossless) {  // Algorithm 2's first step: undo the lossless stage, then decompress
    std::vector<uint8_t> R;
    if (!ll_unpack(s, n, P.L.sumdc, P.raw_total, &R)) return EFORMAT;
    rc = decompress_impl<T>(R.data(), R.size(), field, status, flips, nflips, rep);
    if (rep) rep->compressed_bytes = P.total;
    return rc;
  }
  const Geom& g = P.g;
  orc_report r;
  std::memset(&r, 0, sizeof(r));
  r.blocks = g.nb;
  r.eb_abs = P.eb;
  r.compressed_bytes = P.total;
  r.regression_blocks = P.n_reg;
  r.unpredictable_points = P.n_unpred;
  // per-block offsets by prefix sums; the group table must agree with them
  std::vector<uint64_t> pay_off(g.nb), un_off(g.nb);
  std::vector<int64_t> reg_idx(g.nb);
  uint64_t pay = 0, un = 0, rg = 0;
  for (uint64_t b = 0; b < g.nb; ++b) {
    if (b % kGroup == 0) {
      uint64_t gi = b / kGroup;
      if (get<uint64_t>(s, P.L.groups + 24 * gi) != pay || get<uint64_t>(s, P.L.groups + 24 * gi + 8) != un ||
          get<uint64_t>(s, P.L.groups + 24 * gi + 16) != rg)
        return EFORMAT;
    }
    pay_off[b] = pay;
    un_off[b] = un;
    bool isreg = (get<uint32_t>(s, P.L.bitmap + 4 * (b / 32)) >> (b % 32)) & 1u;
    reg_idx[b] = isreg ? (int64_t)rg : -1;
    pay += get<uint16_t>(s, P.L.sizes + 2 * b);
    un += get<uint16_t>(s, P.L.ucounts + 2 * b);
    rg += isreg ? 1 : 0;
  }
  if (pay != P.payload_bytes || un != P.n_unpred || rg != P.n_reg) return EFORMAT;

  // Algorithm 2: decompress every block
  std::vector<std::vector<T>> dec(g.nb);
  std::vector<uint64_t> sums(g.nb);
  std::vector<uint8_t> ok(g.nb);
  for (uint64_t b = 0; b < g.nb; ++b) {
    uint64_t org[3];
    uint32_t e[3];
    block_box(g, b, org, e);
    dec[b].assign((uint64_t)e[0] * e[1] * e[2], (T)0);
    ok[b] = decompress_block<T>(P, s, b, pay_off[b], un_off[b], reg_idx[b], flips, nflips, true, dec[b].data(), &sums[b]);
  }
  // Algorithm 2: check each block against sum_dc, re-execute once on a mismatch
  int result = OK;
  for (uint64_t b = 0; b < g.nb; ++b) {
    uint8_t st = 0;
    if (P.abft) {
      const uint64_t ref = get<uint64_t>(s, P.L.sumdc + 8 * b);
      if (!ok[b] || sums[b] != ref) {
        ok[b] = decompress_block<T>(P, s, b, pay_off[b], un_off[b], reg_idx[b], flips, nflips, false, dec[b].data(), &sums[b]);
        if (ok[b] && sums[b] == ref) {
          st = 1;
          r.decomp_reexec_corrected++;
        } else {
          st = ok[b] ? 2 : 3;
        }
      }
    } else if (!ok[b]) {
      st = 3;
    }
    if (st >= 2) {
      r.uncorrectable_blocks++;
      result = ESDC;
    }
    if (status) status[b] = st;
    uint64_t org[3];
    uint32_t e[3];
    block_box(g, b, org, e);
    uint64_t k = 0;
    if (field)
      for (uint32_t i = 0; i < e[0]; ++i)
        for (uint32_t j = 0; j < e[1]; ++j)
          for (uint32_t l = 0; l < e[2]; ++l) field[global_index(g, org, i, j, l)] = dec[b][k++];
  }
  if (rep) *rep = r;
  return result;
}

}  // namespace

// ---------------------------------------------------------------- exported entry points
extern "C" {

int orc_compress_bound(const orc_params* p, uint64_t* bytes);

int orc_compress(const void* field, const orc_params* p, const orc_flip* flips, int nflips, uint8_t* out,
                 uint64_t cap, uint64_t* out_bytes, orc_report* rep) {
  if (!p || !out) return EINVAL_;
  if (p->dtype > 1 || p->encoding > 3) return EINVAL_;
  if (!(p->encoding & 2)) {
    if (p->dtype == 0) return compress_impl<float>((const float*)field, p, flips, nflips, out, cap, out_bytes, rep);
    return compress_impl<double>((const double*)field, p, flips, nflips, out, cap, out_bytes, rep);
  }
  // the stream without the lossless stage first, then the stage over it
  uint64_t bound = 0;
  if (orc_compress_bound(p, &bound)) return EINVAL_;
  std::vector<uint8_t> R(bound);
  uint64_t nR = 0;
  orc_report r;
  int rc = p->dtype == 0 ? compress_impl<float>((const float*)field, p, flips, nflips, R.data(), bound, &nR, &r)
                         : compress_impl<double>((const double*)field, p, flips, nflips, R.data(), bound, &nR, &r);
  if (rc) return rc;
  Parsed P;
  if (parse(R.data(), nR, &P)) return EFORMAT;
  std::vector<uint8_t> S;
  ll_pack(R.data(), nR, P.L.sumdc, (uint8_t)(p->encoding & 1), &S);
  if (S.size() > cap) return ECAPACITY;
  std::memcpy(out, S.data(), S.size());
  r.compressed_bytes = S.size();
  if (out_bytes) *out_bytes = S.size();
  if (rep) *rep = r;
  return OK;
}

// Worst case: every point unpredictable and coded with kMaxLen bits, every block regression.
// Compact encoding: each point may also carry a whole value and each block 4 coefficients of
// at most 38 bits.
// The lossless stage can add up to 2 bytes per coded byte plus its tables and states.
int orc_compress_bound(const orc_params* p, uint64_t* bytes) {
  Geom g;
  if (!p || !make_geom(p, &g)) return EINVAL_;
  const bool compact = (p->encoding & 1) != 0;
  Layout L = make_layout(g, p->abft != 0, compact, p->quant_bins ? p->quant_bins : 65536, g.nb, g.N);
  const uint64_t bits = compact ? (uint64_t)g.P * (kMaxLen + 8 * (g.dtype ? 8 : 4)) + 4 * 38 : (uint64_t)g.P * kMaxLen;
  uint64_t b = L.payload + g.nb * ((bits + 7) / 8);
  if (p->encoding & 2) {
    const uint64_t n = b - L.sumdc, nchunks = (n + kLLChunk - 1) / kLLChunk;
    b = L.sumdc + 512 + 4 * nchunks + 16 + 2 * n + nchunks * (4 * kLLWays + 4);
  }
  *bytes = b;
  return OK;
}

int orc_read_header(const uint8_t* s, uint64_t n, orc_params* p, uint64_t* total) {
  Parsed P;
  if (n < kHeader || std::memcmp(s, "SDSZ", 4) != 0) return EFORMAT;
  int rc = parse(s, n, &P);
  if (rc) return rc;
  if (p) *p = P.p;
  if (total) *total = P.total;
  return OK;
}

int orc_decompress(const uint8_t* stream, uint64_t n, void* field, uint8_t* status, const orc_flip* flips, int nflips,
                   orc_report* rep) {
  if (!stream) return EINVAL_;
  if (n < kHeader) return EFORMAT;
  uint8_t dtype = stream[6];
  if (dtype == 0) return decompress_impl<float>(stream, n, (float*)field, status, flips, nflips, rep);
  if (dtype == 1) return decompress_impl<double>(stream, n, (double*)field, status, flips, nflips, rep);
  return EFORMAT;
}

// ---- pieces exposed for pinning the oracle against closed forms and brute force ----

void orc_checksum_words(const uint32_t* w, uint64_t n, uint64_t* sum, uint64_t* isum) { checksum_words(w, n, sum, isum); }

int orc_locate_and_repair(uint32_t* w, uint64_t n, uint64_t sum0, uint64_t isum0, uint64_t maxval) {
  return locate_and_repair(w, n, sum0, isum0, maxval);
}

void orc_huffman_lengths(const uint64_t* hist, uint32_t nsym, uint8_t* len) { huffman_lengths(hist, nsym, len); }

// Canonical codes for given lengths (code_of[s] for every symbol).
void orc_canonical_codes(const uint8_t* len, uint32_t nsym, uint32_t* code_of) {
  Canon c;
  std::vector<uint32_t> co;
  canon_from_lengths(len, nsym, &c, &co);
  for (uint32_t s = 0; s < nsym; ++s) code_of[s] = co[s];
}

// Regression coefficients of one block of values (row-major, extents ext[0..ndim-1]).
int orc_regression(const void* v, uint32_t dtype, uint32_t ndim, const uint32_t* ext, float* coef) {
  uint32_t e[3] = {1, 1, 1};
  for (uint32_t a = 0; a < ndim; ++a) e[3 - ndim + a] = ext[a];
  if (dtype == 0) return regression_coefficients<float>((const float*)v, e, (int)ndim, coef) ? 1 : 0;
  return regression_coefficients<double>((const double*)v, e, (int)ndim, coef) ? 1 : 0;
}

// One block of Algorithm 1's prediction loop with a given absolute bound: codes, reconstructed values
// (through sum_dc), coefficients, predictor flag. Used for sampled checks on large fields.
int orc_compress_block(const void* field, const orc_params* p, double eb_abs, uint64_t b, uint16_t* codes,
                       void* coef, uint8_t* is_reg, uint64_t* sums /* sum_q, isum_q, sum_dc */, uint64_t* n_points) {
  Ctx c;
  if (!make_geom(p, &c.g) || b >= c.g.nb) return EINVAL_;
  c.bins = p->quant_bins;
  c.R = p->quant_bins / 2;
  c.abft = p->abft != 0;
  c.predictor_mode = (int)p->predictor;
  c.compact = p->encoding == 1;
  uint64_t sum_in = 0, isum_in = 0;
  auto run = [&](auto* f, auto tag) -> int {
    typedef decltype(tag) T;
    const T eb = (T)eb_abs;
    const T inv2 = (T)(1.0 / (2.0 * (double)eb));
    BlockResult<T> r;
    Ctx c2 = c;
    c2.abft = false;  // no stored input checksums to verify against
    Prep pr = prepare_block<T>(c2, (const T*)f, b);
    if (c2.compact) quantize_prep<T>(c2, (const T*)f, b, eb, &pr);
    compress_block<T>(c2, (const T*)f, b, eb, inv2, sum_in, isum_in, pr, &r);
    std::memcpy(codes, r.code.data(), 2 * r.code.size());
    std::memcpy(coef, r.coef, sizeof(T) * 4);
    *is_reg = r.regression ? 1 : 0;
    sums[0] = r.sum_q;
    sums[1] = r.isum_q;
    sums[2] = r.sum_dc;
    *n_points = r.code.size();
    return OK;
  };
  if (p->dtype == 0) return run((const float*)field, 0.0f);
  return run((const double*)field, 0.0);
}

// Compact encoding, for pinning: the value an unpredictable point x decompresses to at the
// absolute bound eb (both of the dtype); returns the mantissa bits kept.
int orc_truncate_unpredictable(const void* x, uint32_t dtype, double eb, void* out) {
  if (dtype == 0) {
    const float v = *(const float*)x, e = (float)eb;
    *(float*)out = truncate_unpredictable<float>(v, bound_exponent<float>(e));
    return kept_mantissa_bits<float>(v, bound_exponent<float>(e));
  }
  const double v = *(const double*)x;
  *(double*)out = truncate_unpredictable<double>(v, bound_exponent<double>(eb));
  return kept_mantissa_bits<double>(v, bound_exponent<double>(eb));
}

// Compact encoding, for pinning: coefficient a (ndim = intercept) of a block geometry with
// edges block[0..ndim-1] at the absolute bound eb (of the dtype) as an integer k and its
// dequantized dtype value; returns 0 when it cannot be stored (the block uses Lorenzo).
int orc_quantize_coefficient(float c, uint32_t dtype, uint32_t ndim, const uint32_t* block, double eb, uint32_t a,
                             int32_t* k, void* deq) {
  orc_params p;
  std::memset(&p, 0, sizeof(p));
  p.ndim = ndim;
  p.dtype = dtype;
  for (uint32_t d = 0; d < ndim; ++d) {
    p.dims[d] = block[d];
    p.block[d] = block[d];
  }
  Geom g;
  if (!make_geom(&p, &g) || a > ndim) return -1;
  const double E = dtype == 0 ? (double)(float)eb : eb;
  const CoefSteps qs = coef_steps(g, E);
  if (!quantize_coef(c, qs.inv[a], k)) return 0;
  if (dtype == 0) *(float*)deq = dequantize_coef<float>(*k, qs.step[a]);
  else *(double*)deq = dequantize_coef<double>(*k, qs.step[a]);
  return 1;
}

// Lossless stage, for pinning: frequencies of a byte histogram; one chunk coded and decoded.
void orc_ll_frequencies(const uint64_t* cnt, uint16_t* f) { ll_frequencies(cnt, f); }

uint64_t orc_ll_encode(const uint8_t* in, uint32_t n, const uint16_t* f, uint8_t* out, uint64_t cap) {
  uint32_t c[257];
  ll_cumulative(f, c);
  std::vector<uint8_t> o;
  ll_encode_chunk(in, n, f, c, &o);
  if (o.size() > cap) return 0;
  std::memcpy(out, o.data(), o.size());
  return o.size();
}

void orc_ll_decode(const uint8_t* in, uint64_t len, uint32_t n, const uint16_t* f, uint8_t* out) {
  uint32_t c[257];
  ll_cumulative(f, c);
  std::vector<uint8_t> sym(kLLM, 0);
  for (int b = 0; b < 256; ++b)
    for (uint32_t q = c[b]; q < c[b + 1] && q < kLLM; ++q) sym[q] = (uint8_t)b;
  ll_decode_chunk(in, len, n, f, c, sym.data(), out);
}

// Predictor selection, for pinning (Algorithm 1, "sample and estimate"): the sample
// membership of every point of a block of extents ext[0..ndim-1] (row-major, 1 = sampled);
// returns the number of sampled points.
uint64_t orc_sample_mask(uint32_t ndim, const uint32_t* ext, uint8_t* mask) {
  uint32_t e[3] = {1, 1, 1};
  for (uint32_t a = 0; a < ndim; ++a) e[3 - ndim + a] = ext[a];
  uint64_t k = 0, n = 0;
  for (uint32_t i = 0; i < e[0]; ++i)
    for (uint32_t j = 0; j < e[1]; ++j)
      for (uint32_t l = 0; l < e[2]; ++l, ++k) {
        mask[k] = sample_row((int)ndim, i, j, e) ? 1 : 0;
        n += mask[k];
      }
  return n == sample_points((int)ndim, e) ? n : ~0ull;
}

// The two estimates of one block for given fp32 coefficients.
void orc_selection_estimates(const void* v, uint32_t dtype, uint32_t ndim, const uint32_t* ext, const float* coef,
                             float* Ereg, float* Elor) {
  uint32_t e[3] = {1, 1, 1};
  for (uint32_t a = 0; a < ndim; ++a) e[3 - ndim + a] = ext[a];
  if (dtype == 0) selection_estimates<float>((const float*)v, e, (int)ndim, coef, Ereg, Elor);
  else selection_estimates<double>((const double*)v, e, (int)ndim, coef, Ereg, Elor);
}

// The indicator: 1 = regression.
int orc_select_regression(float Ereg, float Elor, uint64_t S, uint32_t ndim, float eb) {
  return select_regression(Ereg, Elor, S, (int)ndim, eb) ? 1 : 0;
}

// The value-range relative bound of the field, as the compressor computes it.
double orc_error_bound(const void* field, const orc_params* p) {
  Geom g;
  if (!make_geom(p, &g)) return -1.0;
  if (p->eb_mode == 0) return p->dtype ? (double)(double)p->eb : (double)(float)p->eb;
  auto run = [&](auto* f) -> double {
    typedef std::remove_const_t<std::remove_pointer_t<decltype(f)>> T;
    bool any = false;
    T mn = 0, mx = 0;
    for (uint64_t n = 0; n < g.N; ++n) {
      T x = f[n];
      if (!std::isfinite(x)) continue;
      if (!any) { mn = mx = x; any = true; }
      if (x < mn) mn = x;
      if (x > mx) mx = x;
    }
    double ebd = p->eb;
    if (any && mx > mn) ebd = p->eb * ((double)mx - (double)mn);
    return (double)(T)ebd;
  };
  if (p->dtype == 0) return run((const float*)field);
  return run((const double*)field);
}

}  // extern "C"
