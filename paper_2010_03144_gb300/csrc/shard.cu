// Sharded compression: one field split into slabs of whole block rows along its slowest axis,
// each slab on its own GPU, written as the stream a single call writes for the whole field,
// byte for byte. The blocks are independent (Sec. 5.1 of the paper), so a slab's blocks
// compress exactly as they do inside the field once the slabs agree on the three things that
// span the field: the value range (for the value-range relative bound), the code histogram
// (for the one Huffman code of the field) and the running totals of payload bytes,
// unpredictable values and regression blocks (for where each block's data goes). Each stage
// below ends where one of those exchanges is needed; the caller makes the exchange (a
// collective over its ranks) and passes the result to the next stage.
#include <algorithm>
#include <cstddef>
#include <cstring>

#include "host.h"

namespace sdcsz {
namespace {

// The slab's parameters: the field's, with axis 0 cut to block rows [b0, b1).
int slab_params(const sdcsz_params* p_field, uint64_t b0, uint64_t b1, sdcsz_params* p_slab, Geo* g_field, Geo* g_slab,
                uint64_t* boff) {
  if (!p_field) return SDCSZ_EINVAL;
  int rc = make_geo(p_field, g_field);
  if (rc) return rc;
  if (g_field->lossless) return SDCSZ_EINVAL;  // the lossless stage codes the whole stream at once
  const int a0 = 3 - g_field->ndim;            // the slowest axis in the padded geometry
  const uint64_t B = g_field->B[a0], d0 = g_field->d[a0];
  if (b0 >= b1 || b1 > g_field->nbd[a0]) return SDCSZ_EINVAL;
  *p_slab = *p_field;
  p_slab->block[0] = (uint32_t)B;
  p_slab->dims[0] = std::min(b1 * B, d0) - b0 * B;
  rc = make_geo(p_slab, g_slab);
  if (rc) return rc;
  *boff = b0 * (g_field->nb / g_field->nbd[a0]);  // the field's index of the slab's first block
  return SDCSZ_OK;
}

struct Ctx {
  sdcsz_params ps;
  Geo gf, gs;
  uint64_t boff;
  Ws w;
  Launch L;
};

int setup(const sdcsz_params* p_field, uint64_t b0, uint64_t b1, void* d_ws, size_t ws_bytes, void* stream,
          Ctx* c) {
  int rc = slab_params(p_field, b0, b1, &c->ps, &c->gf, &c->gs, &c->boff);
  if (rc) return rc;
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255)) return SDCSZ_EINVAL;
  const WsPlan plan = plan_ws(c->gs);
  if (ws_bytes < plan.total) return SDCSZ_ECAPACITY;
  c->w = bind_ws(d_ws, plan);
  c->L.stream = static_cast<cudaStream_t>(stream);
  c->L.sms = sm_count();
  cudaGetLastError();
  return SDCSZ_OK;
}

int finish(const Ctx& c, State* h) {
  if (cudaGetLastError() != cudaSuccess) return SDCSZ_ECUDA;
  int rc = read_state(c.w.st, c.L.stream, h);
  if (rc) return rc;
  return map_error(h->error);
}

}  // namespace
}  // namespace sdcsz

using namespace sdcsz;

extern "C" int sdcsz_shard_workspace_size(const sdcsz_params* p_field, uint64_t slab_b0, uint64_t slab_b1,
                                          size_t* bytes) {
  sdcsz_params ps;
  Geo gf, gs;
  uint64_t boff;
  const int rc = slab_params(p_field, slab_b0, slab_b1, &ps, &gf, &gs, &boff);
  if (rc) return rc;
  if (!bytes) return SDCSZ_EINVAL;
  *bytes = plan_ws(gs).total;
  return SDCSZ_OK;
}

extern "C" int sdcsz_shard_prep(const void* d_slab, const sdcsz_params* p_field, uint64_t slab_b0, uint64_t slab_b1,
                                void* d_ws, size_t ws_bytes, uint64_t* range_keys, void* stream) {
  Ctx c;
  int rc = setup(p_field, slab_b0, slab_b1, d_ws, ws_bytes, stream, &c);
  if (rc) return rc;
  if (!d_slab || !range_keys) return SDCSZ_EINVAL;
  const Ws& w = c.w;
  if (cudaMemsetAsync(w.st, 0, sizeof(State), c.L.stream) != cudaSuccess) return SDCSZ_ECUDA;
  if (cudaMemsetAsync(w.hist, 0, 8 * (size_t)c.gs.bins, c.L.stream) != cudaSuccess) return SDCSZ_ECUDA;
  const size_t ngroups = (c.gs.nb + kGroup - 1) / kGroup;
  if (cudaMemsetAsync(w.gt, 0, 8 * group_total_words(ngroups), c.L.stream) != cudaSuccess) return SDCSZ_ECUDA;
  {
    NvtxRange r("sdcsz shard prep");
    launch_prep(d_slab, c.gs, w, c.L);
  }
  State h;
  if (cudaGetLastError() != cudaSuccess) return SDCSZ_ECUDA;
  rc = read_state(w.st, c.L.stream, &h);
  if (rc) return rc;
  range_keys[0] = h.min_key;  // both keys grow with the range: a maximum over the slabs is the field's
  range_keys[1] = h.max_key;
  return SDCSZ_OK;
}

extern "C" int sdcsz_shard_predict(const void* d_slab, const sdcsz_params* p_field, uint64_t slab_b0,
                                   uint64_t slab_b1, void* d_ws, size_t ws_bytes, const uint64_t* field_range_keys,
                                   uint64_t* counts, void** d_hist, void* stream) {
  Ctx c;
  int rc = setup(p_field, slab_b0, slab_b1, d_ws, ws_bytes, stream, &c);
  if (rc) return rc;
  if (!d_slab || !field_range_keys || !counts) return SDCSZ_EINVAL;
  const Ws& w = c.w;
  // the field's range replaces the slab's (and the slab's own bound, with any error it raised)
  struct {
    unsigned long long min_key, max_key;
    unsigned int k1_done, error;
  } head = {field_range_keys[0], field_range_keys[1], 0u, 0u};
  static_assert(offsetof(State, min_key) == 0 && offsetof(State, error) == 20, "State layout");
  if (cudaMemcpyAsync(w.st, &head, sizeof(head), cudaMemcpyHostToDevice, c.L.stream) != cudaSuccess) return SDCSZ_ECUDA;
  {
    NvtxRange r("sdcsz shard predict");
    launch_bound(c.gf, w.st, c.L);
    if (c.gs.nb) launch_predict(d_slab, c.gs, w, nullptr, 0, c.L);
  }
  State h;
  rc = finish(c, &h);
  if (rc) return rc;
  counts[0] = h.n_reg;
  counts[1] = h.n_unpred;
  counts[2] = h.uncorrectable;
  if (d_hist) *d_hist = static_cast<void*>(w.hist);
  return SDCSZ_OK;
}

extern "C" int sdcsz_shard_encode(const sdcsz_params* p_field, uint64_t slab_b0, uint64_t slab_b1, void* d_ws,
                                  size_t ws_bytes, const uint64_t* field_counts, int header, void* d_out,
                                  size_t out_cap, uint64_t* totals, void* stream) {
  Ctx c;
  int rc = setup(p_field, slab_b0, slab_b1, d_ws, ws_bytes, stream, &c);
  if (rc) return rc;
  if (!field_counts || !d_out || !totals || out_cap < (size_t)kHeaderBytes) return SDCSZ_EINVAL;
  const Ws& w = c.w;
  // the code table and the layout are the field's: its counts go where the codebook reads them
  const unsigned long long fc[2] = {field_counts[0], field_counts[1]};
  static_assert(offsetof(State, n_unpred) == offsetof(State, n_reg) + 8, "State layout");
  if (cudaMemcpyAsync(&w.st->n_reg, fc, sizeof(fc), cudaMemcpyHostToDevice, c.L.stream) != cudaSuccess)
    return SDCSZ_ECUDA;
  uint8_t* out = static_cast<uint8_t*>(d_out);
  Shard sh;
  std::memset(&sh, 0, sizeof(sh));
  sh.on = 1;
  sh.header = header ? 1 : 0;
  sh.boff = c.boff;
  {
    NvtxRange r("sdcsz shard codebook + encode");
    launch_codebook(c.gf, w, header ? out : nullptr, out_cap, c.L);
    launch_encode_shard_blocks(c.gs, w, out, out_cap, sh, c.L);
  }
  State h;
  rc = finish(c, &h);
  if (rc) return rc;
  // the slab's totals from the super-group words the encoder summed (payload bytes;
  // unpredictables << 17 | regression blocks)
  const uint64_t ngroups = (c.gs.nb + kGroup - 1) / kGroup, nsuper = (ngroups + kSuper - 1) / kSuper;
  unsigned long long sg[2 * 64];
  uint64_t pay = 0, reg = 0;
  for (uint64_t q0 = 0; q0 < nsuper; q0 += 64) {
    const uint64_t n = std::min<uint64_t>(64, nsuper - q0);
    if (cudaMemcpyAsync(sg, w.gt + ngroups + 2 * q0, 16 * n, cudaMemcpyDeviceToHost, c.L.stream) != cudaSuccess)
      return SDCSZ_ECUDA;
    if (cudaStreamSynchronize(c.L.stream) != cudaSuccess) return SDCSZ_ECUDA;
    for (uint64_t q = 0; q < n; ++q) {
      pay += sg[2 * q];
      reg += sg[2 * q + 1] & 0x1ffffull;
    }
  }
  totals[0] = pay;
  totals[1] = h.n_unpred_enc;
  totals[2] = reg;
  totals[3] = h.uncorrectable;
  return SDCSZ_OK;
}

extern "C" int sdcsz_shard_assemble(const sdcsz_params* p_field, uint64_t slab_b0, uint64_t slab_b1, void* d_ws,
                                    size_t ws_bytes, const uint64_t* prefix, const uint64_t* field_totals,
                                    int header, void* d_out, size_t out_cap, size_t* out_bytes,
                                    sdcsz_report* report, void* stream) {
  Ctx c;
  int rc = setup(p_field, slab_b0, slab_b1, d_ws, ws_bytes, stream, &c);
  if (rc) return rc;
  if (!prefix || !field_totals || !d_out) return SDCSZ_EINVAL;
  Shard sh;
  std::memset(&sh, 0, sizeof(sh));
  sh.on = 1;
  sh.header = header ? 1 : 0;
  sh.boff = c.boff;
  for (int q = 0; q < 3; ++q) sh.pre[q] = prefix[q];
  for (int q = 0; q < 4; ++q) sh.tot[q] = field_totals[q];
  {
    NvtxRange r("sdcsz shard assemble");
    launch_encode_shard_assemble(c.gs, c.w, static_cast<uint8_t*>(d_out), out_cap, sh, c.L);
  }
  State h;
  rc = finish(c, &h);
  if (rc) return rc;
  if (report) fill_report(h, c.gs.nb, report);
  if (out_bytes) *out_bytes = (size_t)h.total_bytes;
  return SDCSZ_OK;
}
