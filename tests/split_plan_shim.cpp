// Test-only C entry point over the library's split-contraction plan
// (paper_2010_04559_gb300/csrc/split_plan.hpp), compiled by
// tests/test_split_arithmetic.py so that the plan the library runs is the one
// whose exactness the tests check.  Not part of libamgt.
#include "split_plan.hpp"

extern "C" {

// bits, nsl and the passes of split_plan(K): pass p has scale index d[p] and
// gemms [start[p], start[p+1]) of (i, j, beta).  Returns the number of passes
// (-1 if a buffer of `cap` entries is too small).
int shim_split_plan(int K, int* bits, int* nsl, int* d, int* start, int* gi, int* gj,
                    float* beta, int cap) {
  const amgt::SplitPlan p = amgt::split_plan(K);
  *bits = p.bits;
  *nsl = p.nsl;
  int n = 0;
  for (size_t q = 0; q < p.passes.size(); ++q) {
    if ((int)q >= cap) return -1;
    d[q] = p.passes[q].d;
    start[q] = n;
    for (const amgt::SplitGemm& g : p.passes[q].gemms) {
      if (n >= cap) return -1;
      gi[n] = g.i, gj[n] = g.j, beta[n] = g.beta;
      ++n;
    }
  }
  if ((int)p.passes.size() >= cap) return -1;
  start[p.passes.size()] = n;
  return (int)p.passes.size();
}

}  // extern "C"
