// Build-time generator: the nonzero pattern of the nodal differentiation matrices Dr, Ds that
// make_refelem() computes, written as constexpr tables.  The kernels test these bits with
// compile-time indices, so structural zeros (39 % of Dr and Ds at p = 2, 46 % at p = 4) cost no
// FP64 instruction; the values themselves stay in constant memory, uploaded at run time.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>

#include "internal.h"

namespace slt {
void set_error(const std::string&) {}
void fail(int, const std::string& msg) {
  std::fprintf(stderr, "refgen: %s\n", msg.c_str());
  std::exit(1);
}
}  // namespace slt

int main() {
  std::printf("// generated at build time by refgen.cpp from make_refelem(); do not edit\n#pragma once\n");
  std::printf("#include <stdint.h>\nnamespace slt {\n");
  for (int which = 0; which < 2; ++which) {
    std::printf("__host__ __device__ constexpr uint32_t %s_nz(int p, int i) {\n", which ? "ds" : "dr");
    for (int p = 1; p <= 4; ++p) {
      slt::RefElem R = slt::make_refelem(p);
      const std::vector<double>& D = which ? R.Ds : R.Dr;
      double mx = 0;
      for (double x : D) mx = std::fmax(mx, std::fabs(x));
      std::printf("  if (p == %d) {\n    constexpr uint32_t m[%d] = {", p, R.Np);
      for (int i = 0; i < R.Np; ++i) {
        uint32_t bits = 0;
        for (int j = 0; j < R.Np; ++j)
          if (std::fabs(D[i * R.Np + j]) > 1e-12 * mx) bits |= 1u << j;
        std::printf("%s0x%xu", i ? ", " : "", bits);
      }
      std::printf("};\n    return m[i];\n  }\n");
    }
    std::printf("  return 0xffffffffu;\n}\n");
  }
  std::printf("}  // namespace slt\n");
  return 0;
}
