// check.cuh - global-memory accessors of the kernels, and the LBM_CHECK
// debug build behind them (a stand-in for a device memory checker).
//
// Every load, store and atomic of a kernel on global memory goes through the
// accessors below. In the normal build they are the plain operations and
// compile to the same code as writing them out. Built with -DLBM_CHECK
// (liblbm_check.so), each access is first tested against the table of
// buffers its launch was given: byte range [lo, hi), read and/or write
// permission, and natural alignment of the access. An access that fits no
// permitted range, or is misaligned, is NOT performed (a load returns zero,
// a store or atomic is dropped); it is counted, and the address, size and
// kind of the first one are kept in a device record that the host reads with
// lbm_check_status(). Nothing traps and nothing hangs.
//
// Tables: each launcher states the buffers of its launch with
// LBM_CHECK_TABLE(stream, ranges...), which (check build only) launches a
// one-thread kernel on the same stream that copies the table, passed by
// value, into this translation unit's table; stream order makes it visible
// to the launch that follows, and inside a captured CUDA graph it becomes a
// node of its own. The table lives in the translation unit (static), so a
// check build checks launches of one stream at a time: calls on several
// streams at once may see one another's tables.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#ifdef LBM_CHECK
#include <initializer_list>
#endif

namespace lbm {

enum : unsigned { kChkRead = 1u, kChkWrite = 2u, kChkRW = 3u };

// The refused-access record (device memory; one per process).
struct CheckRecord {
  unsigned long long count;  // accesses refused since the last reset
  unsigned long long first;  // address of the first refused access
  unsigned int first_bytes;  // its size in bytes
  unsigned int first_kind;   // kChkRead / kChkWrite / kChkRW it needed
};

constexpr int kCheckRanges = 200;  // the table is a kernel parameter (< 4 KB)

struct CheckTable {
  int n;
  unsigned perm[kCheckRanges];
  unsigned long long lo[kCheckRanges], hi[kCheckRanges];
  CheckRecord *rec;
};

// One buffer of a launch: `bytes` from p, with permission `perm`.
struct CheckRange {
  const void *p;
  size_t bytes;
  unsigned perm;
};
inline CheckRange chk_r(const void *p, size_t bytes) { return {p, bytes, kChkRead}; }
inline CheckRange chk_w(const void *p, size_t bytes) { return {p, bytes, kChkWrite}; }
inline CheckRange chk_rw(const void *p, size_t bytes) { return {p, bytes, kChkRW}; }

#ifdef LBM_CHECK

static __device__ CheckTable s_check_table;

static __global__ void k_check_set(const CheckTable t) { s_check_table = t; }

// `align`: the alignment the access needs (a power of two).
static __device__ __noinline__ bool check_access(const void *p, unsigned bytes, unsigned align,
                                                 unsigned need) {
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  const CheckTable &t = s_check_table;
  if ((a & (align - 1)) == 0) {
    for (int r = 0; r < t.n; ++r)
      if (a >= t.lo[r] && a + bytes <= t.hi[r] && (t.perm[r] & need) == need) return true;
  }
  if (t.rec != nullptr && atomicAdd(&t.rec->count, 1ull) == 0ull) {
    t.rec->first = a;
    t.rec->first_bytes = bytes;
    t.rec->first_kind = need;
  }
  return false;
}
#define LBM_CHK(p, bytes, align, need) ::lbm::check_access((p), (bytes), (align), (need))

// The process's record (allocated on first use; lbm_capi.cu).
CheckRecord *check_record();
// Ranges narrowed by this many bytes at their end (lbm_check_narrow).
size_t check_narrow_bytes();

// Null or empty ranges are left out; a range given twice gets the union of
// its permissions. More than kCheckRanges distinct ranges is a build error
// of the caller, reported as cudaErrorInvalidValue.
static inline cudaError_t check_table(cudaStream_t s, const CheckRange *rs, int nr) {
  CheckTable t{};
  const size_t narrow = check_narrow_bytes();
  for (int k = 0; k < nr; ++k) {
    const CheckRange &r = rs[k];
    if (r.p == nullptr || r.bytes == 0) continue;
    const unsigned long long lo = reinterpret_cast<unsigned long long>(r.p);
    const unsigned long long hi = lo + (r.bytes > narrow ? r.bytes - narrow : 0);
    int j = 0;
    while (j < t.n && !(t.lo[j] == lo && t.hi[j] == hi)) ++j;
    if (j == t.n) {
      if (t.n == kCheckRanges) return cudaErrorInvalidValue;
      t.lo[j] = lo;
      t.hi[j] = hi;
      ++t.n;
    }
    t.perm[j] |= r.perm;
  }
  t.rec = check_record();
  k_check_set<<<1, 1, 0, s>>>(t);
  return cudaGetLastError();
}
static inline cudaError_t check_table(cudaStream_t s, std::initializer_list<CheckRange> rs) {
  return check_table(s, rs.begin(), (int)rs.size());
}
#define LBM_CHECK_TABLE(s, ...) ((void)::lbm::check_table((s), {__VA_ARGS__}))

#else

#define LBM_CHK(p, bytes, align, need) true
#define LBM_CHECK_TABLE(s, ...) ((void)0)

#endif

// ---- accessors ---------------------------------------------------------------
// LBM_LD: plain load; LBM_LDV: volatile load; LBM_LDG: read-only
// (non-coherent) path; LBM_LDCG: L2 only; LBM_ST: plain store (*p = v);
// LBM_ACC: plain *p += v; LBM_STCS: streaming store; LBM_ATOMIC_ADD,
// LBM_ATOMIC_OR: atomicAdd, atomicOr; LBM_VALID(p): whether the whole object
// at p may be read (for structures read field by field through a reference).
// In the normal build each is the bare expression it names, textually, so
// that the kernels compile exactly as written out (forwarding stores through
// even inlined functions changed ptxas's register allocation).
#ifdef LBM_CHECK
template <class T>
__device__ __forceinline__ T chk_ld(const T *p) {
  return LBM_CHK(p, sizeof(T), sizeof(T), kChkRead) ? *p : T{};
}
template <class T>
__device__ __forceinline__ T chk_ldv(const T *p) {
  return LBM_CHK(p, sizeof(T), sizeof(T), kChkRead) ? *reinterpret_cast<const volatile T *>(p)
                                                    : T{};
}
template <class T>
__device__ __forceinline__ T chk_ldg(const T *p) {
  return LBM_CHK(p, sizeof(T), sizeof(T), kChkRead) ? __ldg(p) : T{};
}
template <class T>
__device__ __forceinline__ T chk_ldcg(const T *p) {
  return LBM_CHK(p, sizeof(T), sizeof(T), kChkRead) ? __ldcg(p) : T{};
}
template <class T, class U>
__device__ __forceinline__ void chk_st(T *p, U v) {
  if (LBM_CHK(p, sizeof(T), sizeof(T), kChkWrite)) *p = v;
}
template <class T, class U>
__device__ __forceinline__ void chk_acc(T *p, U v) {
  if (LBM_CHK(p, sizeof(T), sizeof(T), kChkRW)) *p += v;
}
template <class T>
__device__ __forceinline__ void chk_stcs(T *p, T v) {
  if (LBM_CHK(p, sizeof(T), sizeof(T), kChkWrite)) __stcs(p, v);
}
template <class T>
__device__ __forceinline__ T chk_atomic_add(T *p, T v) {
  return LBM_CHK(p, sizeof(T), sizeof(T), kChkRW) ? atomicAdd(p, v) : T{};
}
template <class T>
__device__ __forceinline__ T chk_atomic_or(T *p, T v) {
  return LBM_CHK(p, sizeof(T), sizeof(T), kChkRW) ? atomicOr(p, v) : T{};
}
template <class T>
__device__ __forceinline__ bool chk_valid(const T *p) {
  return LBM_CHK(p, sizeof(T), alignof(T), kChkRead);
}
#define LBM_LD(p) ::lbm::chk_ld(p)
#define LBM_LDV(p) ::lbm::chk_ldv(p)
#define LBM_LDG(p) ::lbm::chk_ldg(p)
#define LBM_LDCG(p) ::lbm::chk_ldcg(p)
#define LBM_ST(p, v) ::lbm::chk_st((p), (v))
#define LBM_ACC(p, v) ::lbm::chk_acc((p), (v))
#define LBM_STCS(p, v) ::lbm::chk_stcs((p), (v))
#define LBM_ATOMIC_ADD(p, v) ::lbm::chk_atomic_add((p), (v))
#define LBM_ATOMIC_OR(p, v) ::lbm::chk_atomic_or((p), (v))
#define LBM_VALID(p) ::lbm::chk_valid(p)
#else
#define LBM_LD(p) (*(p))
#define LBM_LDV(p) (*(const volatile decltype(+*(p)) *)(p))
#define LBM_LDG(p) __ldg(p)
#define LBM_LDCG(p) __ldcg(p)
#define LBM_ST(p, v) ((void)(*(p) = (v)))
#define LBM_ACC(p, v) ((void)(*(p) += (v)))
#define LBM_STCS(p, v) __stcs((p), (v))
#define LBM_ATOMIC_ADD(p, v) atomicAdd((p), (v))
#define LBM_ATOMIC_OR(p, v) atomicOr((p), (v))
#define LBM_VALID(p) true
#endif

}  // namespace lbm
