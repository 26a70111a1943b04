// Plan of the split FP64 contraction on the tensor cores: digit width,
// slices and GEMM passes for an inner dimension K.  Plain host C++ (no CUDA),
// included by capi.cu and compiled by the CPU tests, which check it against
// the exactness conditions below.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

namespace amgt {

// Slice width and GEMM passes of the split FP64 contraction for inner
// dimension K (kernels_split64.cu): `bits` b is the largest (at most 7, so
// that digits up to 2^7 are exact in BF16) with K 2^(2b) <= 2^24, the range
// of exact FP32 integers; nsl = ceil(50 / b) slices keep 50 bits of each
// operand, and the products of slices (i, j) with i + j = d < nsl are taken.
// Leading diagonals d < dt = ceil(26 / b): the pairs are grouped so that the
// sum of their bounds K D_i D_j (D_0 = 2^b, D_i = 2^(b-1)) stays within 2^24,
// each group accumulated exactly on the tensor cores (beta = 1) and then in
// FP64.  Trailing diagonals d >= dt: one Horner pass from d = nsl - 1 down
// to dt in FP32 (the first product of each diagonal takes beta = 2^-b); its
// rounding is 2^-24 of a sum 2^(-b dt) <= 2^-26 below the leading term.
// bits = 0: the split form does not apply.
struct SplitGemm {
  int i, j;
  float beta;
};
struct SplitPass {
  std::vector<SplitGemm> gemms;
  int d;  // the pass is accumulated into y with the scale 2^(-b (d + 2))
};
struct SplitPlan {
  int bits = 0, nsl = 0;
  std::vector<SplitPass> passes;
};

inline SplitPlan split_plan(int K) {
  SplitPlan p;
  int b = 7;
  const double lim = std::ldexp(1.0, 24);
  while (b > 0 && (double)K * std::ldexp(1.0, 2 * b) > lim) --b;
  if (b < 2) return p;
  p.bits = b;
  p.nsl = (50 + b - 1) / b;
  const int dt = std::min(p.nsl, (26 + b - 1) / b);
  auto D = [&](int i) { return std::ldexp(1.0, i == 0 ? b : b - 1); };
  for (int d = 0; d < dt; ++d) {
    SplitPass cur{{}, d};
    double acc = 0.0;
    for (int i = 0; i <= d; ++i) {
      const double bound = (double)K * D(i) * D(d - i);
      if (!cur.gemms.empty() && acc + bound > lim) {
        p.passes.push_back(cur);
        cur = SplitPass{{}, d};
        acc = 0.0;
      }
      cur.gemms.push_back({i, d - i, cur.gemms.empty() ? 0.0f : 1.0f});
      acc += bound;
    }
    p.passes.push_back(cur);
  }
  if (dt < p.nsl) {
    SplitPass tail{{}, dt};
    for (int d = p.nsl - 1; d >= dt; --d)
      for (int i = 0; i <= d; ++i) {
        const float beta =
            tail.gemms.empty() ? 0.0f : (i == 0 ? std::ldexp(1.0f, -b) : 1.0f);
        tail.gemms.push_back({i, d - i, beta});
      }
    p.passes.push_back(tail);
  }
  return p;
}

}  // namespace amgt
