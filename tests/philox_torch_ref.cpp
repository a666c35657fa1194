// Black-box reference for the oracle's Philox4x32-10: PyTorch's header-only
// at::philox_engine (ATen/core/PhiloxRNGEngine.h), an implementation written
// independently of this repository.  Reads lines "key64 subseq64 offset64"
// and prints the four 32-bit outputs of the block at counter
// (offset lo, offset hi, subseq lo, subseq hi) under that key.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cinttypes>
#include <cstdio>

int main() {
  unsigned long long key, sub, off;
  while (std::scanf("%llu %llu %llu", &key, &sub, &off) == 3) {
    at::philox_engine e(key, sub, off);
    uint32_t a = e(), b = e(), c = e(), d = e();
    std::printf("%" PRIu32 " %" PRIu32 " %" PRIu32 " %" PRIu32 "\n", a, b, c, d);
  }
  return 0;
}
