// K5's two-pass decoder of large cube blocks (see decode_wave.cuh), both encodings and both
// precisions.
#include "decode.cuh"
#include "decode_wave.cuh"

namespace sdcsz {

bool launch_decode_wave(const uint8_t* s, uint64_t nbytes, const Hdr& h, void* field, uint8_t* status, State* st,
                        uint8_t* wave_ws, const Launch& L) {
  // the shapes whose one-pass decoding would take the generic kernel (one thread per block with
  // its Lorenzo plane in shared memory): 16^3, and 10^3 and 12^3 in float64
  if (!wave_decode_ws_bytes(h.g) || !field) return false;
  if (h.g.dtype == 0 ? kdec::has_fast<float>(h.g) : kdec::has_fast<double>(h.g)) return false;
  if (h.g.dtype == 0) {
    return h.g.enc ? kdec::try_wave_decode<float, true>(s, nbytes, h, static_cast<float*>(field), status, st, wave_ws, L)
                   : kdec::try_wave_decode<float, false>(s, nbytes, h, static_cast<float*>(field), status, st, wave_ws,
                                                         L);
  }
  return h.g.enc ? kdec::try_wave_decode<double, true>(s, nbytes, h, static_cast<double*>(field), status, st, wave_ws, L)
                 : kdec::try_wave_decode<double, false>(s, nbytes, h, static_cast<double*>(field), status, st, wave_ws,
                                                        L);
}

}  // namespace sdcsz
