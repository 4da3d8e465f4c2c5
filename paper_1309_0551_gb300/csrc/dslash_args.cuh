// Arguments of one single-lattice half Dslash launch (k_dslash, k_dslash_rw).
#pragma once

#include "lqcd_internal.cuh"

struct DslashKArgs {
  const char* gauge;
  size_t blk_bytes;
  Geom G;
  int out_par;
  const void* in;
  void* out;
  size_t rhs_stride;
  int nrhs;
  const void* w1;
  double a1;
  const void* w2;
  double a2;
  double c;
  int reduce;
  Reducer red;
  int pdl;     // host side only: launch with programmatic dependent launch
  unsigned int* status;   // the context's device status word (bounded waits that gave up)
};
