// Device side of the persistent far chains (hmat_chain.cu: FP32, mixed mode;
// hmat_chain64.cu: FP64): the bounded dependency waits of an item and the completion
// count it publishes. Tickets are handed out in list order and every dependency names
// an earlier item, so the unfinished item with the lowest ticket always has its inputs.
// A producer's thread 0 publishes after a CTA barrier and a device-scope fence; a
// consumer's thread 0 reads with acquire semantics before a CTA barrier, which orders
// the other threads' operand reads after it. Every wait is bounded: after limit_ns it
// latches HMAT_ETIMEOUT in the status word and sets the launch's abort flag, and every
// CTA then stops taking tickets.
#pragma once

#include <cuda_runtime.h>

#include "hmat_internal.h"

namespace hmat {

static __device__ __forceinline__ uint64_t chain_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

static __device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 only: wait until *cnt >= need (need <= 0: nothing to wait for). False when the
// launch aborted or the wait ran out (which latches HMAT_ETIMEOUT and aborts the launch).
static __device__ bool chain_wait(const int32_t* cnt, int need, const ChainLaunch& l, int* status, uint64_t* t0) {
  if (need <= 0) return true;
  uint32_t nap = 32;  // back off, so that many waiting CTAs do not crowd the counters' cache lines
  for (uint32_t i = 0;; ++i) {
    if (ld_acquire(cnt) >= need) return true;
    if ((i & 7) == 7) {
      if (*(volatile int32_t*)l.abort_flag) return false;
      const uint64_t t = chain_timer();
      if (*t0 == 0) {
        *t0 = t;
      } else if (t - *t0 > l.limit_ns) {
        atomicCAS(status, 0, (int)HMAT_ETIMEOUT);
        atomicExch(l.abort_flag, 1);
        return false;
      }
    }
    __nanosleep(nap);
    nap = nap < 2048 ? 2 * nap : 2048;
  }
}

// The dependencies of one item (thread 0).
static __device__ bool chain_deps(const ChainSync& m, const ChainItem& it, const ChainLaunch& l) {
  const int n = m.n_nodes;
  const int32_t* e_up = m.expect;
  const int32_t* e_cpl = m.expect + n;
  const int32_t* e_dn = m.expect + 2 * n;
  const int32_t* e_lvl = m.expect + 3 * n;
  const int32_t* c_up = m.ctr;
  const int32_t* c_cpl = m.ctr + n;
  const int32_t* c_dn = m.ctr + 2 * n;
  const int32_t* c_lvl = m.ctr + 3 * n;
  const int nct = m.n_ct;
  uint64_t t0 = 0;
  auto need = [&](const int32_t* e, int node) { return e[node] > 0 ? e[node] * nct + l.extra : 0; };
  // self-test: the root never has a basis, so its upward counter stays 0 and this wait runs out
  if (l.extra > 0 && !chain_wait(c_up, l.extra, l, m.status, &t0)) return false;
  const int a = it.node;
  switch (it.kind) {
    case CK_UP:
      if ((l.waits & kWaitUp) && a < m.first_leaf)
        for (int c = 2 * a + 1; c <= 2 * a + 2; ++c)
          if (!chain_wait(c_up + c, need(e_up, c), l, m.status, &t0)) return false;
      return true;
    case CK_CPL:
      if (l.waits & kWaitLevel)
        return chain_wait(c_lvl + it.level, need(e_lvl, it.level), l, m.status, &t0);
      return true;
    case CK_DN:
    case CK_LEAF:
      if (l.waits & kWaitCpl) {
        if (!chain_wait(c_cpl + a, need(e_cpl, a), l, m.status, &t0)) return false;
        if (it.kind == CK_DN)
          for (int c = 2 * a + 1; c <= 2 * a + 2; ++c)
            if (!chain_wait(c_cpl + c, need(e_cpl, c), l, m.status, &t0)) return false;
      }
      if ((l.waits & kWaitDn) && a >= 1) {
        const int p = (a - 1) / 2;
        if (!chain_wait(c_dn + p, need(e_dn, p), l, m.status, &t0)) return false;
      }
      return true;
  }
  return true;
}

// Thread 0: item ii of a member's list, checked against the sizes it indexes (the item
// array, the tile array, the tree's nodes) before any of them is read through it; false
// (nothing read) for an inconsistent index.
static __device__ __forceinline__ bool chain_item_ok(const ChainItem* items, int64_t ii, int32_t n_items,
                                                     int32_t n_tiles, int32_t n_nodes, ChainItem* out) {
  if (ii < 0 || ii >= n_items) return false;
  const ChainItem it = items[ii];
  if (it.tile < 0 || it.tile >= n_tiles || it.node < 0 || it.node >= n_nodes || it.kind > CK_LEAF) return false;
  *out = it;
  return true;
}

// Thread 0, after the CTA barrier that ends the item's tile: count it complete.
static __device__ __forceinline__ void chain_done(const ChainSync& m, const ChainItem& it) {
  if (it.kind == CK_LEAF) return;  // nothing waits for a leaf item
  __threadfence();
  const int n = m.n_nodes;
  switch (it.kind) {
    case CK_UP:
      atomicAdd(m.ctr + it.node, 1);
      atomicAdd(m.ctr + 3 * n + it.level, 1);
      break;
    case CK_CPL: atomicAdd(m.ctr + n + it.node, 1); break;
    case CK_DN: atomicAdd(m.ctr + 2 * n + it.node, 1); break;
    default: break;
  }
}

}  // namespace hmat
