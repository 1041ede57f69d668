// Exact summation of doubles (fixed-point accumulator over the whole
// exponent range, rounded once).  Every Pauli coefficient the builder emits
// is the correctly rounded value of the exact sum of its contributions, so
// the table does not depend on the order in which terms are generated.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace gocp {

void ExactSum::clear() {
  std::memset(limb_, 0, sizeof(limb_));
  adds_ = 0;
  special_ = 0.0;
  has_special_ = false;
}

void ExactSum::normalize(int64_t* l) const {
  for (int i = 0; i < kLimbs - 1; ++i) {
    int64_t carry = l[i] >> 32;           // floor division by 2^32
    l[i] -= carry * ((int64_t)1 << 32);   // now in [0, 2^32)
    l[i + 1] += carry;
  }
}

void ExactSum::add(double v) {
  if (v == 0.0) return;
  if (!std::isfinite(v)) {
    special_ += v;
    has_special_ = true;
    return;
  }
  int e = 0;
  double m = std::frexp(std::fabs(v), &e);          // |v| = m 2^e, m in [0.5, 1)
  uint64_t mant = (uint64_t)std::ldexp(m, 53);      // |v| = mant 2^(e-53)
  int pos = e - 53 + kOffset;                       // bit index of mant's lowest bit
  if (pos < 0) {                                    // subnormal: low bits are zero
    mant >>= -pos;
    pos = 0;
  }
  int li = pos / 32, sh = pos % 32;
  unsigned __int128 w = (unsigned __int128)mant << sh;
  int64_t d0 = (int64_t)(uint64_t)(w & 0xffffffffu);
  int64_t d1 = (int64_t)(uint64_t)((w >> 32) & 0xffffffffu);
  int64_t d2 = (int64_t)(uint64_t)((w >> 64) & 0xffffffffu);
  if (v < 0) { d0 = -d0; d1 = -d1; d2 = -d2; }
  limb_[li] += d0;
  limb_[li + 1] += d1;
  limb_[li + 2] += d2;
  if ((++adds_ & 0xffffff) == 0) normalize(limb_);
}

double ExactSum::round() const {
  if (has_special_) return special_;
  int64_t l[kLimbs];
  std::memcpy(l, limb_, sizeof(l));
  normalize(l);
  bool neg = l[kLimbs - 1] < 0;
  if (neg) {
    for (int i = 0; i < kLimbs; ++i) l[i] = -l[i];
    normalize(l);
  }
  int top = -1;
  for (int i = kLimbs - 1; i >= 0; --i)
    if (l[i] != 0) { top = i; break; }
  if (top < 0) return 0.0;
  auto bit = [&](int k) -> int { return k < 0 ? 0 : (int)((l[k / 32] >> (k % 32)) & 1); };
  int msb = 63 - __builtin_clzll((unsigned long long)l[top]);
  int p = top * 32 + msb;
  int lo = p - 52 > kMinBit ? p - 52 : kMinBit;
  uint64_t mant = 0;
  for (int k = p; k >= lo; --k) mant = (mant << 1) | (uint64_t)bit(k);
  int rbit = bit(lo - 1);
  bool sticky = false;
  int below = lo - 1;                                // bits [0, below) are sticky
  for (int i = 0; i < below / 32 && !sticky; ++i) sticky = l[i] != 0;
  if (!sticky && below > 0) {
    int i = below / 32, r = below % 32;
    if (r) sticky = (l[i] & (((int64_t)1 << r) - 1)) != 0;
  }
  if (rbit && (sticky || (mant & 1))) mant += 1;
  double out = std::ldexp((double)mant, lo - kOffset);
  return neg ? -out : out;
}

}  // namespace gocp
