// fs_col_tma.cuh -- column groups staged into shared memory by bulk copies
// (FP32; power-of-two column lengths with register tile 16, 3 x 2^k / 5 x 2^k
// lengths with their family's tile, 24 / 20).  Used by the standalone
// persistent column kernel, inlined into the batch kernel (powers of two) and
// called from it (the other two families, fs_mixed_f32.cu).
#pragma once
#include "fs_tma.cuh"
#include "fs_units.cuh"

namespace fs {

// The work on one staged group: columns g .. g+cc-1 (below g_end) in `cur`
// ([column][L], unpadded), which then doubles as the FFT exchange area.
// (rho, t): the thread's column in the group and its slot; adv: an advance
// (no forward transform); dst: the work spectrum; tw: the length-L twiddles.
template <int L>
__device__ __forceinline__ void col_tma_group(const Desc &d, int g, int g_end, int cc, cx<float> *cur, int rho,
                                              int t, bool adv, cx<float> *dst, const cx<float> *tw) {
  constexpr int E = mx_e(L) ? mx_e(L) : 16, Tseg = L / E;
  const int a = g + rho;
  const bool active = rho < cc && a < g_end;
  cx<float> u[E];
  if (active) {
#pragma unroll
    for (int s = 0; s < E; ++s) u[s] = cur[rho * L + t + Tseg * s];
  } else {
#pragma unroll
    for (int s = 0; s < E; ++s) u[s] = zero_cx<float>();
  }
  const XLayout lay{rho * L, 1};
  if (!adv) fft_ct_from<float, E, L, 1, 1, 0>(u, cur, lay.base, active, t, tw);
  if (!adv && d.st_out_u && active) {  // keep the forward spectrum
    cx<float> *ou = reinterpret_cast<cx<float> *>(d.st_out_u) + (size_t)a * L;
#pragma unroll
    for (int s = 0; s < E; ++s) ou[t + Tseg * s] = u[s];
  }
  if (d.op != OP_FORWARD) {
    if (active) col_op_single<float, E>(d, op_ctx<float>(d, a), t, Tseg, u);
    // no barrier here: the transform's first exchange store into `cur`
    // comes after its own barrier, which every read of `cur` above precedes
    fft_ct_from<float, E, L, 1, 1, 0>(u, cur, lay.base, active, t, tw);
    if (active) {
      cx<float> *o = dst + (size_t)a * L;
#pragma unroll
      for (int s = 0; s < E; ++s) o[t + Tseg * s] = conj(u[s]);
    }
  }
}
// the same out of line (a caller that keeps the copy loop's state in few registers)
template <int L>
__device__ __noinline__ void col_tma_group_ool(const Desc &d, int g, int g_end, int cc, cx<float> *cur, int rho,
                                               int t, bool adv, cx<float> *dst, const cx<float> *tw) {
  col_tma_group<L>(d, g, g_end, cc, cur, rho, t, adv, dst, tw);
}

// A column group is cc consecutive columns a = g .. g+cc-1: one contiguous run
// of the x-frequency-major spectrum, so a single bulk copy (cp.async.bulk,
// completion on an mbarrier) stages a whole group into shared memory.  The
// groups g = g_first, g_first + g_step, ... below g_end are walked with two
// buffers: the NEXT group is copied in while the current one is transformed
// (the current buffer doubles as the FFT exchange area).  The standalone
// kernel walks groups blockIdx.x*CC, += gridDim.x*CC over all columns; a batch
// work unit walks its own consecutive groups.  Single field only (the
// two-field wave variants use k_col_p2).
//
// ph holds the parity of the next completion of each barrier (bit k for
// bars[k]) and carries across calls from the same CTA; every call starts on
// buffer 0.  Returns false when a copy did not land within kTmaWaitNs (the
// device error word is set, and the copy still in flight has been waited for,
// again bounded).
template <int L, int CC, bool OOL = false>
__device__ __forceinline__ bool col_tma_groups(const Desc &d, int g_first, int g_step, int g_end, int cc_rt,
                                               cx<float> *buf0, cx<float> *buf1, uint64_t *bars, uint32_t &ph,
                                               int *s_abort) {
  constexpr int E = mx_e(L) ? mx_e(L) : 16, Tseg = L / E;
  const int cc = CC ? CC : cc_rt;
  const int tid = threadIdx.x;
  const int rho = tid / Tseg, t = tid - rho * Tseg;
  const bool adv = (d.op == OP_DIFF_ADV || d.op == OP_WAVE_ADV);
  const cx<float> *src = reinterpret_cast<const cx<float> *>(adv ? d.st_u : d.work_u);
  cx<float> *dst = reinterpret_cast<cx<float> *>(d.work_u);
  const cx<float> *tw = reinterpret_cast<const cx<float> *>(d.tw_y);
  auto issue = [&](cx<float> *b, uint64_t *bar, int g) {
    const int nc = min(cc, g_end - g);
    const uint32_t bytes = (uint32_t)(nc * L * sizeof(cx<float>));
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(b, src + (size_t)g * L, bytes, bar);
  };
  // earlier generic accesses of this CTA to the buffers (a previous unit)
  // are ordered before the bulk writes into them
  fence_proxy_async_smem();
  __syncthreads();
  if (tid == 0) {
    *s_abort = 0;
    // a solve's work spectrum may come from other CTAs of this launch (seen
    // through the batch's acquire): order it before the bulk copies read it
    if (!adv) fence_proxy_async_global();
    if (g_first < g_end) issue(buf0, &bars[0], g_first);
  }
  __syncthreads();
  int i = 0;
  for (int g = g_first; g < g_end; g += g_step, ++i) {
    const int k = i & 1;
    cx<float> *cur = k ? buf1 : buf0;
    cx<float> *nxt = k ? buf0 : buf1;
    const bool more = g + g_step < g_end;
    if (tid == 0 && more) issue(nxt, &bars[k ^ 1], g + g_step);
    // every thread observes the copy's completion itself (bounded)
    if (!mbar_wait_bounded(&bars[k], (ph >> k) & 1u, kTmaWaitNs)) {
      atomicExch(&g_fs_dev_error, FS_DEV_ERR_TMA_TIMEOUT);
      *s_abort = 1;
    }
    ph ^= 1u << k;
    __syncthreads();
    if (*s_abort) {
      // let the copies still in flight land before the CTA leaves (bounded
      // again): this group's, if it is the one that timed out (its phase
      // parity is the one just flipped in ph), and the next group's
      if (tid == 0) {
        mbar_wait_bounded(&bars[k], ((ph >> k) & 1u) ^ 1u, kTmaWaitNs);
        if (more) mbar_wait_bounded(&bars[k ^ 1], (ph >> (k ^ 1)) & 1u, kTmaWaitNs);
      }
      return false;
    }
    if constexpr (OOL)
      col_tma_group_ool<L>(d, g, g_end, cc, cur, rho, t, adv, dst, tw);
    else
      col_tma_group<L>(d, g, g_end, cc, cur, rho, t, adv, dst, tw);
    fence_proxy_async_smem();
    __syncthreads();
  }
  return true;
}

}  // namespace fs
