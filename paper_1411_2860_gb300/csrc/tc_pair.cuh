// Cluster-multicast forms used by the CTA pairs of the reduced GEMMs: a TMA
// load delivered to both CTAs of a cluster, and an MMA commit that arrives on
// the same mbarrier in both.  The tensor maps these loads read cover this
// GPU's own memory only.  Included only when PJ_CTA_PAIRS is set (tc.cuh): the
// library built for several GPUs, one process each, compiles none of this.
#pragma once

#include "tc.cuh"

#if !PJ_CTA_PAIRS
#error "tc_pair.cuh is part of the CTA-pair build only"
#endif

namespace pj {

// The same copy delivered to every CTA of the cluster in `mask`, at the same
// shared-memory offset, each signalling its own mbarrier at `bar`'s offset.
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

// As umma_commit, arriving on the mbarrier at `bar`'s offset in every CTA of `mask`.
__device__ __forceinline__ void umma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

}  // namespace pj
