// State-indexed power lookup construction (Sec. 4.1), host side: Liberty-
// style state patterns ("when" conditions that fix some pins and leave the
// others don't-care) expanded into the dense state-indexed arrays that
// gtp_load_library takes.  Each pattern is binary-encoded over the cell's pin
// order; its don't-care pins are enumerated and every complete assignment
// names one array entry.  An entry takes the item of the first pattern (in
// list order) that covers it; entries no pattern covers take the default.
#include <cstring>
#include <vector>

#include "../../include/gtpower.h"

namespace {

// Every subset of `free` (bit mask), including the empty one, in turn.
template <class F>
void for_each_subset(uint32_t free, F f) {
  uint32_t sub = 0u;
  for (;;) {
    f(sub);
    if (sub == free) break;
    sub = (sub - free) & free;  // next subset in increasing order
  }
}

// Side-input index of input state S for an event on `pin`: the other input
// pins' bits, compacted in pin order.
uint32_t compact_side(uint32_t S, int pin) {
  const uint32_t low = S & ((1u << pin) - 1u);
  const uint32_t high = (S >> (pin + 1)) << pin;
  return low | high;
}

}  // namespace

extern "C" int gtp_sipl_expand(int32_t n_in, int32_t n_slew, int32_t n_load, int32_t n_int_pat, const int32_t* int_pin,
                               const int32_t* int_edge, const uint32_t* int_care, const uint32_t* int_val,
                               const float* int_tab, const float* int_default, int32_t n_leak_pat,
                               const uint32_t* leak_care, const uint32_t* leak_val, const float* leak_pw,
                               float leak_default, float* e_int, float* p_leak) {
  if (n_in < 1 || n_in + 1 > GTP_MAX_PINS || n_slew < 2 || n_slew > GTP_MAX_AXIS || n_load < 2 ||
      n_load > GTP_MAX_AXIS || n_int_pat < 0 || n_leak_pat < 0)
    return GTP_ERANGE;
  if (!int_default || !e_int || !p_leak) return GTP_EINVAL;
  if (n_int_pat > 0 && (!int_pin || !int_edge || !int_care || !int_val || !int_tab)) return GTP_EINVAL;
  if (n_leak_pat > 0 && (!leak_care || !leak_val || !leak_pw)) return GTP_EINVAL;
  const uint32_t in_mask = (1u << n_in) - 1u, all_mask = (2u << n_in) - 1u;
  for (int k = 0; k < n_int_pat; ++k) {
    const int p = int_pin[k];
    if (p < 0 || p >= n_in || int_edge[k] < -1 || int_edge[k] > 1) return GTP_EINVAL;
    const uint32_t allowed = in_mask & ~(1u << p);  // the other input pins
    if ((int_care[k] & ~allowed) || (int_val[k] & ~int_care[k])) return GTP_EINVAL;
  }
  for (int k = 0; k < n_leak_pat; ++k)
    if ((leak_care[k] & ~all_mask) || (leak_val[k] & ~leak_care[k])) return GTP_EINVAL;

  const size_t T = (size_t)n_slew * n_load;
  const uint32_t n_side = 1u << (n_in - 1);
  // internal power: per (pin, edge), the side states each pattern covers
  std::vector<char> filled((size_t)n_in * 2 * n_side, 0);
  for (int k = 0; k < n_int_pat; ++k) {
    const int p = int_pin[k];
    const uint32_t free = in_mask & ~(1u << p) & ~int_care[k];
    for (int e = 0; e < 2; ++e) {
      if (int_edge[k] >= 0 && int_edge[k] != e) continue;
      for_each_subset(free, [&](uint32_t sub) {
        const uint32_t side = compact_side(int_val[k] | sub, p);
        const size_t entry = ((size_t)p * 2 + e) * n_side + side;
        if (filled[entry]) return;
        filled[entry] = 1;
        std::memcpy(e_int + entry * T, int_tab + (size_t)k * T, sizeof(float) * T);
      });
    }
  }
  for (size_t entry = 0; entry < filled.size(); ++entry)
    if (!filled[entry]) std::memcpy(e_int + entry * T, int_default + (entry / n_side) * T, sizeof(float) * T);
  // leakage: the full states (output included) each pattern covers
  std::vector<char> lf((size_t)all_mask + 1, 0);
  for (int k = 0; k < n_leak_pat; ++k)
    for_each_subset(all_mask & ~leak_care[k], [&](uint32_t sub) {
      const uint32_t s = leak_val[k] | sub;
      if (lf[s]) return;
      lf[s] = 1;
      p_leak[s] = leak_pw[k];
    });
  for (uint32_t s = 0; s <= all_mask; ++s)
    if (!lf[s]) p_leak[s] = leak_default;
  return GTP_OK;
}
