// Host build of the float32 voxel-mean helper used by the map build kernel.
// Reads "hi_bits lo_bits n" (hex, hex, decimal) per line and prints
// "ok result_bits" per line, so that a test can compare the helper with exact
// rational arithmetic.  Build: g++ -O2 -ffp-contract=off -std=c++17.
#include <cstdio>

#include "../../paper_2202_00242_gb300/csrc/vgicp_mean.h"

int main() {
  unsigned hb, lb, n;
  while (std::scanf("%x %x %u", &hb, &lb, &n) == 3) {
    float hi, lo;
    std::memcpy(&hi, &hb, 4);
    std::memcpy(&lo, &lb, 4);
    bool ok = false;
    const volatile float rN = 1.0f / (float)n;  // RN32(1 / n)
    const float q = vgicp::mean_rn32(hi, lo, n, rN, ok);
    unsigned qb;
    std::memcpy(&qb, &q, 4);
    std::printf("%d %08x\n", ok ? 1 : 0, qb);
  }
  return 0;
}
