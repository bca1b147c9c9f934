// Double-buffered tile streaming with TMA bulk copies (sm_90+ / sm_103a).
//
// A persistent CTA walks the element tiles tile = blockIdx.x, + gridDim.x, ...
// Every input of a tile is a contiguous block of global memory (element-major
// layouts), so one cp.async.bulk per block moves it into shared memory, and
// one mbarrier per buffer counts the bytes (complete_tx).  While the CTA
// computes tile k from buffer k&1, the copies of tile k+1 fill the other
// buffer.  Only thread 0 issues copies and waits with a bound; the outcome is
// broadcast through shared memory so that all threads leave together if a
// wait ever times out (then the kernel raises the timeout flag and returns
// after a bounded wait for its own copies in flight).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dgx {

constexpr int MAXBLK = 16;  // input blocks per tile

// One input block: element e's part starts at base + e * bpe bytes.
struct Blk {
  const void* base;
  uint32_t bpe;  // bytes per element (multiple of 16)
};

struct TileIn {
  Blk b[MAXBLK];
  int nb;
  uint32_t bytes_per_elem;  // sum of bpe
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait (each try_wait suspends for a hardware-defined interval).
constexpr uint32_t WAIT_POLLS = 1u << 22;  // default bound
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t polls = WAIT_POLLS) {
  for (uint32_t it = 0; it < polls; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}

// Issue the copies of elements [e0, e0 + nel) of every block into dst.
// Block k occupies T * bpe_k bytes of the buffer (tile-size stride, so a
// partial last tile uses the start of each region).  Thread 0 only.
__device__ __forceinline__ void tile_issue(const TileIn& in, int e0, int nel, int T, unsigned char* dst,
                                           uint64_t* bar) {
  fence_proxy_async();  // earlier generic-proxy reads of dst are ordered before the async writes
  mbar_expect_tx(bar, in.bytes_per_elem * (uint32_t)nel);
  uint32_t off = 0;
  for (int k = 0; k < in.nb; ++k) {
    bulk_g2s(dst + off, (const unsigned char*)in.b[k].base + (size_t)e0 * in.b[k].bpe, in.b[k].bpe * (uint32_t)nel,
             bar);
    off += in.b[k].bpe * (uint32_t)T;
  }
}

// Shared state of the pipeline (lives in static shared memory of the kernel).
struct PipeState {
  uint64_t bar[2];
  int abort;
};

}  // namespace dgx

namespace dgx {
// Host helper: append a block if it can be streamed (16-byte multiple and
// 16-byte aligned base); returns false otherwise.
inline bool tilein_add(TileIn& in, const void* base, size_t bpe) {
  if (in.nb >= MAXBLK || bpe % 16 != 0 || ((uintptr_t)base & 15) != 0 || bpe > 0xffffffffu) return false;
  in.b[in.nb].base = base;
  in.b[in.nb].bpe = (uint32_t)bpe;
  in.bytes_per_elem += (uint32_t)bpe;
  ++in.nb;
  return true;
}
}  // namespace dgx
