// check.cuh - global-memory accessors of the kernels, and the LBM_CHECK
// debug build behind them (a stand-in for a device memory checker).
//
// Every load, store and atomic of a kernel on global memory goes through the
// accessors below. In the normal build each is the bare operation (the
// read-only and L2-only loads with the prefetch hint of the next section),
// written out by the preprocessor, so no check costs anything. Built with -DLBM_CHECK
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
// Ranges longer than this many bytes are narrowed by it at their end
// (lbm_check_narrow).
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
    const unsigned long long hi = lo + (r.bytes > narrow ? r.bytes - narrow : r.bytes);
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

// ---- L2 prefetch-hinted loads -------------------------------------------------
// Read-only (non-coherent) and L2-only loads that also ask L2 for the whole
// 256-byte block around the address (the .L2::256B prefetch-size
// qualifier). The kernels stream every plane row by row: a warp's loads span
// 64 to 256 bytes, and the hint fetches the block the next warps of the row
// will read in the same request. Measured on GB300: +1.7% for the 16-bit
// step at 384^3 (pair loads of 128 bytes per warp; the 128-byte hint changes
// nothing), +0.6 to 1.4% for the one-node FP32 kernels (batched forward and
// reverse sequences, adjoint step), no change for the FP32 two-node step
// (its pair loads already span 256 bytes). DRAM bytes and instruction counts
// are unchanged. Types other than the ones below use the plain intrinsics.
__device__ __forceinline__ float ldg_pf(const float *p) {
  float v;
  asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ldg_pf(const float2 *p) {
  float2 v;
  asm("ld.global.nc.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
template <class T>
__device__ __forceinline__ T ldg_pf(const T *p) {
  return __ldg(p);
}
__device__ __forceinline__ float ldcg_pf(const float *p) {
  float v;
  asm("ld.global.cg.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
template <class T>
__device__ __forceinline__ T ldcg_pf(const T *p) {
  return __ldcg(p);
}

// ---- accessors ---------------------------------------------------------------
// LBM_LD: plain load; LBM_LDV: volatile load; LBM_LDG: read-only
// (non-coherent) path; LBM_LDCG: L2 only (both with the prefetch hint
// above where the type has one); LBM_ST: plain write-back store (*p = v);
// LBM_ACC: plain *p += v; LBM_ATOMIC_ADD, LBM_ATOMIC_OR: atomicAdd,
// atomicOr; LBM_VALID(p): whether the whole object at p may be read (for
// structures read field by field through a reference).
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
  return LBM_CHK(p, sizeof(T), sizeof(T), kChkRead) ? ldg_pf(p) : T{};
}
template <class T>
__device__ __forceinline__ T chk_ldcg(const T *p) {
  return LBM_CHK(p, sizeof(T), sizeof(T), kChkRead) ? ldcg_pf(p) : T{};
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
#define LBM_ATOMIC_ADD(p, v) ::lbm::chk_atomic_add((p), (v))
#define LBM_ATOMIC_OR(p, v) ::lbm::chk_atomic_or((p), (v))
#define LBM_VALID(p) ::lbm::chk_valid(p)
#else
#define LBM_LD(p) (*(p))
#define LBM_LDV(p) (*(const volatile decltype(+*(p)) *)(p))
#define LBM_LDG(p) ::lbm::ldg_pf(p)
#define LBM_LDCG(p) ::lbm::ldcg_pf(p)
#define LBM_ST(p, v) ((void)(*(p) = (v)))
#define LBM_ACC(p, v) ((void)(*(p) += (v)))
#define LBM_ATOMIC_ADD(p, v) atomicAdd((p), (v))
#define LBM_ATOMIC_OR(p, v) atomicOr((p), (v))
#define LBM_VALID(p) true
#endif

// 16-, 32- and 64-bit raw loads of 16-bit storage (pairs and groups of four
// values), with the prefetch hint, checked like every access.
__device__ __forceinline__ unsigned short ldg_pf_b16(const void *p) {
  if (!LBM_CHK(p, 2u, 2u, kChkRead)) return 0;
  unsigned short v;
  asm("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned ldg_pf_b32(const void *p) {
  if (!LBM_CHK(p, 4u, 4u, kChkRead)) return 0u;
  unsigned v;
  asm("ld.global.nc.L2::256B.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ldg_pf_v2b32(const void *p) {
  if (!LBM_CHK(p, 8u, 8u, kChkRead)) return make_uint2(0u, 0u);
  uint2 v;
  asm("ld.global.nc.L2::256B.v2.b32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}

}  // namespace lbm
