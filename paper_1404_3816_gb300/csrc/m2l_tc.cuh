// Tensor-core M2L of the H^2 product (internal).
#pragma once

#include "hikf_internal.cuh"

namespace hikf {

// every level of one H^2 product in one launch per pass of up to 256 rays
struct M2lTcAll {
  int dim = 2, q = 0, ld = 0, sms = 1, nlev = 0;
  int lev[16];                        // levels, ascending (2 .. L)
  int64_t box0[16], nbox[16];         // first box and box count of each level (contiguous, in order)
  const float* W = nullptr;           // [box][q][ld] multipoles (all levels)
  float* L = nullptr;                 // [box][q][ld] locals (all levels); written for these levels
  const float* kop = nullptr;         // [level - 2][offset][q][q] operators of these levels
  const int64_t* nsrc = nullptr;      // per box (all levels): sources below
  const int64_t* npts = nullptr;      // per box (all levels): points below
  int* err = nullptr;                 // device word, set when a bounded wait times out
  bool autotune = true;               // time the feasible variants once per shape
};

bool m2l_tc_supported(int q, int ld);
Status m2l_tc_all(const M2lTcAll& a, cudaStream_t s);

}  // namespace hikf
