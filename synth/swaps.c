/*
 * swaps.c -- input generation only: applies a list of index-pair swaps to an
 * array, one after another in list order, so that a "sortedness" input with
 * r = 10^9 swaps (Sec. 1's inputs of varying sortedness) takes seconds
 * rather than minutes.  The swap list is drawn by the caller; this code holds
 * none of the sorting method's arithmetic.  The result equals applying the
 * swaps sequentially: the look-ahead below only prefetches cache lines.
 */
#include <stddef.h>
#include <stdint.h>

#define AHEAD 64

void synth_apply_swaps_u32(uint32_t* a, const int64_t* i, const int64_t* j, size_t m) {
  size_t k;
  for (k = 0; k < m; ++k) {
    uint32_t t;
    if (k + AHEAD < m) {
      __builtin_prefetch(&a[i[k + AHEAD]], 1, 0);
      __builtin_prefetch(&a[j[k + AHEAD]], 1, 0);
    }
    t = a[i[k]];
    a[i[k]] = a[j[k]];
    a[j[k]] = t;
  }
}

void synth_apply_swaps_u64(uint64_t* a, const int64_t* i, const int64_t* j, size_t m) {
  size_t k;
  for (k = 0; k < m; ++k) {
    uint64_t t;
    if (k + AHEAD < m) {
      __builtin_prefetch(&a[i[k + AHEAD]], 1, 0);
      __builtin_prefetch(&a[j[k + AHEAD]], 1, 0);
    }
    t = a[i[k]];
    a[i[k]] = a[j[k]];
    a[j[k]] = t;
  }
}
