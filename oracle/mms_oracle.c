/*
 * mms_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * The plain, slow, obviously correct CPU reference for the GPU Multiway
 * Mergesort hot path.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this code; the product library never does.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (Sec. 4 "Multiway Mergesort", Sec. 4.1 "Parallel
 * Partitioning"): the sorted order of N keys under a comparison function.
 * Because the method reaches that result exactly, the oracle is the plain
 * definition written out: a textbook top-down two-way mergesort, stable
 * (on equal keys the merge takes from the left run), so the output is the
 * unique permutation that is non-decreasing in the key order with equal keys
 * kept in input order.  Values (32-bit payloads) move with their keys.
 *
 * Key types: 4-byte and 8-byte unsigned integers (the paper's workloads,
 * Sec. 6.3) and IEEE-754 binary32.  The paper is silent on floats; the
 * reading taken is IEEE-754-2008 totalOrder on bit patterns, written here in
 * sign-magnitude form (not as a bit flip):
 *     -NaN < -inf < ... < -0.0 < +0.0 < ... < +inf < +NaN,
 * NaNs ordered by their payload bits, output bits unchanged.
 *
 * Test hook: oracle_set_mutation() plants one known mistake in the oracle so
 * that the test suite can show its pins catch it.  Mutation 0 (the default)
 * is the correct oracle.
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { KEY_U32 = 0, KEY_U64 = 1, KEY_F32 = 2 };

/* Planted-mistake selector, only for the tests that check the pins. */
enum {
  MUT_NONE = 0,
  MUT_TIES_FROM_RIGHT = 1,   /* merge takes from the right run on equal keys */
  MUT_F32_IGNORE_SIGN = 2,   /* f32 compared as raw unsigned bits */
  MUT_F32_NEG_ASCENDING = 3, /* negative floats ordered by ascending bits */
  MUT_U64_LOW_WORD_ONLY = 4, /* u64 compared on the low 32 bits only */
  MUT_MERGE_DUP_LAST = 5     /* merge writes the left run's last item twice */
};
static int g_mutation = MUT_NONE;

void oracle_set_mutation(int m) { g_mutation = m; }
int oracle_get_mutation(void) { return g_mutation; }

/* ---- key order ---------------------------------------------------------- */

static uint32_t f32_bits(const float* a, size_t i) {
  uint32_t u;
  memcpy(&u, &a[i], sizeof u);
  return u;
}

/* x strictly before y in IEEE-754 totalOrder, sign-magnitude formulation. */
static int f32_total_order_less(uint32_t x, uint32_t y) {
  uint32_t sx = x >> 31, sy = y >> 31;
  if (g_mutation == MUT_F32_IGNORE_SIGN) return x < y;
  if (sx != sy) return sx > sy;             /* the negative one comes first */
  if (sx == 0) return x < y;                /* both positive: ascending */
  if (g_mutation == MUT_F32_NEG_ASCENDING) return x < y;
  return x > y;                             /* both negative: descending bits */
}

/* keys[i] strictly before keys[j] in the key order of key_type. */
int oracle_less(int key_type, const void* keys, size_t i, size_t j) {
  switch (key_type) {
    case KEY_U32: {
      const uint32_t* a = (const uint32_t*)keys;
      return a[i] < a[j];
    }
    case KEY_U64: {
      const uint64_t* a = (const uint64_t*)keys;
      if (g_mutation == MUT_U64_LOW_WORD_ONLY)
        return (uint32_t)a[i] < (uint32_t)a[j];
      return a[i] < a[j];
    }
    case KEY_F32: {
      const float* a = (const float*)keys;
      return f32_total_order_less(f32_bits(a, i), f32_bits(a, j));
    }
    default:
      return 0;
  }
}

/* ---- stable top-down two-way mergesort on an index permutation --------- */

/* Merges the sorted halves idx[lo, mid) and idx[mid, hi) through tmp. */
static void merge_halves(int kt, const void* keys, uint64_t* idx, uint64_t* tmp,
                         size_t lo, size_t mid, size_t hi) {
  size_t i, j, o;
  i = lo;
  j = mid;
  o = lo;
  while (i < mid && j < hi) {
    int take_right;
    if (g_mutation == MUT_TIES_FROM_RIGHT)
      take_right = !oracle_less(kt, keys, idx[i], idx[j]); /* ties -> right */
    else
      take_right = oracle_less(kt, keys, idx[j], idx[i]);  /* ties -> left */
    tmp[o++] = take_right ? idx[j++] : idx[i++];
  }
  while (i < mid) tmp[o++] = idx[i++];
  while (j < hi) tmp[o++] = idx[j++];
  if (g_mutation == MUT_MERGE_DUP_LAST && hi - lo >= 4)
    tmp[hi - 1] = tmp[hi - 2];
  memcpy(idx + lo, tmp + lo, (hi - lo) * sizeof(uint64_t));
}

static void merge_sort_rec(int kt, const void* keys, uint64_t* idx,
                           uint64_t* tmp, size_t lo, size_t hi) {
  size_t mid;
  if (hi - lo < 2) return;
  mid = lo + (hi - lo) / 2;
  merge_sort_rec(kt, keys, idx, tmp, lo, mid);
  merge_sort_rec(kt, keys, idx, tmp, mid, hi);
  merge_halves(kt, keys, idx, tmp, lo, mid, hi);
}

/* The same recursion with its top `depth` levels run as threads: the left
 * half of every such level on a new thread, the right half on this one, then
 * the same merge.  It splits the same ranges and merges them the same way, so
 * its result equals merge_sort_rec's; only the CPU baseline's timing uses it. */
typedef struct {
  int kt;
  const void* keys;
  uint64_t* idx;
  uint64_t* tmp;
  size_t lo, hi;
  int depth;
} sort_task;

static void* merge_sort_task(void* arg);

static void merge_sort_par(const sort_task* t) {
  size_t mid;
  pthread_t th;
  sort_task left, right;
  if (t->depth <= 0 || t->hi - t->lo < ((size_t)1 << 16)) {
    merge_sort_rec(t->kt, t->keys, t->idx, t->tmp, t->lo, t->hi);
    return;
  }
  mid = t->lo + (t->hi - t->lo) / 2;
  left = *t;
  left.hi = mid;
  left.depth = t->depth - 1;
  right = *t;
  right.lo = mid;
  right.depth = t->depth - 1;
  if (pthread_create(&th, NULL, merge_sort_task, &left) != 0) {
    merge_sort_par(&left);                  /* no thread to spare: same work, in order */
    merge_sort_par(&right);
  } else {
    merge_sort_par(&right);
    pthread_join(th, NULL);
  }
  merge_halves(t->kt, t->keys, t->idx, t->tmp, t->lo, mid, t->hi);
}

static void* merge_sort_task(void* arg) {
  merge_sort_par((const sort_task*)arg);
  return NULL;
}

/* perm[p] = input index of the item that lands at output position p. */
int oracle_argsort(int key_type, const void* keys, size_t n, uint64_t* perm) {
  uint64_t* tmp;
  size_t i;
  if (key_type < KEY_U32 || key_type > KEY_F32) return -2;
  for (i = 0; i < n; ++i) perm[i] = i;
  if (n < 2) return 0;
  tmp = (uint64_t*)malloc(n * sizeof(uint64_t));
  if (!tmp) return -1;
  merge_sort_rec(key_type, keys, perm, tmp, 0, n);
  free(tmp);
  return 0;
}

/* oracle_argsort with the recursion's top levels on up to `threads` threads. */
int oracle_argsort_parallel(int key_type, const void* keys, size_t n, uint64_t* perm,
                            int threads) {
  uint64_t* tmp;
  size_t i;
  sort_task t;
  int depth = 0;
  if (key_type < KEY_U32 || key_type > KEY_F32) return -2;
  for (i = 0; i < n; ++i) perm[i] = i;
  if (n < 2) return 0;
  tmp = (uint64_t*)malloc(n * sizeof(uint64_t));
  if (!tmp) return -1;
  while ((1 << depth) < threads && depth < 10) ++depth;
  t.kt = key_type;
  t.keys = keys;
  t.idx = perm;
  t.tmp = tmp;
  t.lo = 0;
  t.hi = n;
  t.depth = depth;
  merge_sort_par(&t);
  free(tmp);
  return 0;
}

static size_t key_bytes(int key_type) { return key_type == KEY_U64 ? 8 : 4; }

/* Sorts keys (and values, when not NULL) in place, stably; threads > 1 runs
 * the recursion's top levels in parallel (same result). */
int oracle_sort_threads(int key_type, void* keys, uint32_t* values, size_t n, int threads) {
  uint64_t* perm;
  unsigned char* kcopy;
  uint32_t* vcopy = NULL;
  size_t kb = key_bytes(key_type), p;
  int rc;
  if (key_type < KEY_U32 || key_type > KEY_F32) return -2;
  if (n < 2) return 0;
  perm = (uint64_t*)malloc(n * sizeof(uint64_t));
  kcopy = (unsigned char*)malloc(n * kb);
  if (values) vcopy = (uint32_t*)malloc(n * sizeof(uint32_t));
  if (!perm || !kcopy || (values && !vcopy)) {
    free(perm);
    free(kcopy);
    free(vcopy);
    return -1;
  }
  rc = threads > 1 ? oracle_argsort_parallel(key_type, keys, n, perm, threads)
                   : oracle_argsort(key_type, keys, n, perm);
  if (rc == 0) {
    memcpy(kcopy, keys, n * kb);
    if (values) memcpy(vcopy, values, n * sizeof(uint32_t));
    for (p = 0; p < n; ++p) {
      memcpy((unsigned char*)keys + p * kb, kcopy + perm[p] * kb, kb);
      if (values) values[p] = vcopy[perm[p]];
    }
  }
  free(perm);
  free(kcopy);
  free(vcopy);
  return rc;
}

/* Sorts keys (and values, when not NULL) in place, stably. */
int oracle_sort(int key_type, void* keys, uint32_t* values, size_t n) {
  return oracle_sort_threads(key_type, keys, values, n, 1);
}
