// Warp-cooperative step kernel shared by both precisions.
//
// A warp owns 32 consecutive particle slots.  Their list entries are
// contiguous in the CSR list, so:
//   A. the lanes walk the warp's flattened entries 32 at a time (coalesced
//      list reads), pre-test each pair for overlap with a cheap conservative
//      test, and append the candidates (entry code and partner slot) to a
//      per-warp queue in shared memory, prefetching their history records
//      into L2; the queue is in entry order, so each particle's contacts are
//      contiguous and in ascending partner index;
//   B. the lanes evaluate the contact law for 32 queued contacts at a time
//      (all lanes busy), write the friction history, and park each contact's
//      force/torque on its own particle in shared memory; then the parked
//      contributions are added to the particles' sums in queue order, one
//      lane per (particle, component) of the batch, the sums kept in shared
//      memory (six independent sequences per particle, so the lanes share the
//      work and every component is summed in the same order as by one lane);
//      A and B alternate in rounds whenever the queue is full, which keeps
//      the order and bounds the shared memory;
//   M. the lanes evaluate the particle-element contacts of the warp's
//      particles 32 candidates at a time and add them in order, as in B;
//   C. each lane integrates its particle.
// The sum of every particle is therefore taken in exactly the order of the
// per-particle loop (ascending partner caller index, then triangle index),
// whatever the launch shape.  Policies supply the precision-specific parts.
#pragma once

#include "dem_internal.cuh"
#include "dem_math.cuh"
#include "dem_step_common.cuh"

namespace dem {

// Warps per block: 4 by default; 8 is the other shape the autotuner can pick
// (dem_params.step_warps).  The resident-block bound of a policy is stated
// for 4-warp blocks and scaled for others, so the threads per SM stay alike.
constexpr int kQueueMax = 512;            // queued contacts per warp and round

template <typename CT>
struct WarpScratch {
  uint32_t seg[33];     // entry prefix of the warp's particles
  uint32_t istart[33];  // queued-contact prefix of the warp's particles
  uint32_t cnt[32];
  uint8_t nlow[32];
  uint16_t qcode[kQueueMax];  // (particle << 6) | entry
  uint32_t qslot[kQueueMax];  // partner slot
  CT contrib[32][6];
  CT acc_h[32][6];  // per-particle sums of phase B (hi words, or the sums)
  CT acc_l[32][6];  // their compensation words (unused by plain sums)
};

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <typename Pol, int Warps>
__global__ void __launch_bounds__(32 * Warps, (Pol::kMinBlocks * 4 / Warps > 0 ? Pol::kMinBlocks * 4 / Warps : 1))
k_step_warp(Ctl* ctl, Params p, StateBufs sb, Lists L, MeshDev mesh, double* forces) {
  using Rec = typename Pol::Rec;
  using Hist = typename Pol::Hist;
  using CT = typename Pol::T;
  __shared__ WarpScratch<CT> smem[Warps];
  if (ctl->status) return;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpScratch<CT>& S = smem[wib];
  const int n = p.n;
  const int w0 = (blockIdx.x * Warps + wib) * 32;
  const int t = w0 + lane;
  const bool valid = t < n;
  const uint32_t ph = ctl->phase & 1u, lph = ctl->lphase & 1u;
  const uint32_t stamp_now = (uint32_t)ctl->step;
  const uint32_t stamp_new = stamp_now + 1u;
  const Rec* P = static_cast<const Rec*>(buf_of(sb.P, ph));
  const Rec* V = static_cast<const Rec*>(buf_of(sb.V, ph));
  const Rec* W = static_cast<const Rec*>(buf_of(sb.W, ph));
  const ListBuf lb = list_of(L, lph);
  Hist* H = static_cast<Hist*>(lb.hpp);

  const uint32_t meta = valid ? lb.meta[t] : 0u;
  const uint32_t nn = meta & 0xffu;
  const uint32_t incl = warp_incl_scan(nn);
  S.seg[lane + 1] = incl;
  if (lane == 0) {
    S.seg[0] = 0;
    S.istart[0] = 0;
  }
  S.nlow[lane] = (uint8_t)((meta >> 8) & 0xffu);
  const uint32_t E = __shfl_sync(full, incl, 31);
  uint32_t base = 0;
  if (w0 < n && lane == 0) base = lb.offs[w0];
  base = __shfl_sync(full, base, 0);

  uint32_t npair = 0;
  typename Pol::Acc acc;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    S.acc_h[lane][c] = CT(0);
    S.acc_l[lane][c] = CT(0);
  }
  uint32_t e0 = 0;
  do {
    S.cnt[lane] = 0;
    __syncwarp();
    // A: overlap pre-test over the warp's flattened entries, queue candidates
    uint32_t qn = 0;
    for (; e0 < E && qn + 32 <= (uint32_t)kQueueMax; e0 += 32) {
      const uint32_t e = e0 + lane;
      bool hit = false;
      uint32_t code = 0, u = 0;
      int tl = 0;
      if (e < E) {
        // the particle owning entry e: largest tl with seg[tl] <= e
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (S.seg[lo + step] <= e) lo += step;
        tl = lo;
        const uint32_t k = e - S.seg[tl];
        u = lb.nbr[base + e];
        // cheap symmetric pre-test; the exact overlap is taken in phase B
        hit = Pol::near(P[w0 + tl], P[u]);
        code = ((uint32_t)tl << 6) | k;
        if (hit) asm volatile("prefetch.global.L2 [%0];" ::"l"(H + base + e));
      }
      const unsigned m = __ballot_sync(full, hit);
      if (hit) {
        const uint32_t pos = qn + __popc(m & ((1u << lane) - 1u));
        S.qcode[pos] = (uint16_t)code;
        S.qslot[pos] = u;
        atomicAdd(&S.cnt[tl], 1u);
      }
      qn += __popc(m);
    }
    __syncwarp();
    const uint32_t icl = warp_incl_scan(S.cnt[lane]);
    S.istart[lane + 1] = icl;
    __syncwarp();

    // B: contact law for 32 queued contacts at a time, then ordered
    // per-particle sums (a queued pair found apart by the exact test
    // contributes zero and keeps no history)
    for (uint32_t i0 = 0; i0 < qn; i0 += 32) {
      const uint32_t i = i0 + lane;
      CT c6[6] = {CT(0), CT(0), CT(0), CT(0), CT(0), CT(0)};
      if (i < qn) {
        const uint32_t code = S.qcode[i];
        const uint32_t u = S.qslot[i];
        const int tl = (int)(code >> 6);
        const uint32_t k = code & 63u;
        const uint32_t e = base + S.seg[tl] + k;
        const bool t_is_i = k >= S.nlow[tl];
        const Rec Pt = P[w0 + tl], Pu = P[u];
        const Rec Vt = V[w0 + tl], Vu = V[u];
        const Rec Wt = W[w0 + tl], Wu = W[u];
        const typename Pol::Aux At = Pol::aux(lb, w0 + tl), Au = Pol::aux(lb, u);
        Hist h = H[e];
        if (Pol::pair(p, t_is_i, t_is_i ? Pt : Pu, t_is_i ? Pu : Pt, t_is_i ? Vt : Vu,
                      t_is_i ? Vu : Vt, t_is_i ? Wt : Wu, t_is_i ? Wu : Wt, t_is_i ? At : Au,
                      t_is_i ? Au : At, h, stamp_now, stamp_new, c6)) {
          H[e] = h;
          ++npair;
        }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) S.contrib[lane][c] = c6[c];
      __syncwarp();
      // the particles with contacts in this batch are pa .. pb (owner of a
      // queue position: largest particle whose range starts at or before it)
      const uint32_t last = (i0 + 32 < qn ? i0 + 32 : qn) - 1u;
      int pa = 0, pb = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        if (S.istart[pa + step] <= i0) pa += step;
        if (S.istart[pb + step] <= last) pb += step;
      }
      const int njobs = (pb - pa + 1) * 6;
      for (int j = lane; j < njobs; j += 32) {
        const int pp = pa + j / 6, c = j % 6;
        const uint32_t ra = S.istart[pp], rb = S.istart[pp + 1];
        const uint32_t a = ra > i0 ? ra : i0;
        const uint32_t b = rb < i0 + 32 ? rb : i0 + 32;
        CT h = S.acc_h[pp][c], l = S.acc_l[pp][c];
        for (uint32_t jj = a; jj < b; ++jj) Pol::Acc::add1(h, l, S.contrib[jj - i0][c]);
        S.acc_h[pp][c] = h;
        S.acc_l[pp][c] = l;
      }
      __syncwarp();
    }
  } while (e0 < E);
  __syncwarp();
  acc.set(S.acc_h[lane], S.acc_l[lane]);

  // M: particle-element contacts of the warp's particles, 32 candidates at a
  // time (all lanes busy), then ordered sums as in B: every lane adds the
  // touching contacts of its own particle in candidate (element index) order
  uint32_t nmesh = 0;
  {
    const uint32_t nt_l = valid ? (meta >> 16) & 0xffu : 0u;
    const uint32_t mincl = warp_incl_scan(nt_l);
    __syncwarp();
    S.seg[lane + 1] = mincl;
    if (lane == 0) S.seg[0] = 0;
    const uint32_t Mt = __shfl_sync(full, mincl, 31);
    __syncwarp();
    const uint32_t my_a = S.seg[lane], my_b = S.seg[lane + 1];
    for (uint32_t c0 = 0; c0 < Mt; c0 += 32) {
      const uint32_t c = c0 + lane;
      CT c6[6] = {CT(0), CT(0), CT(0), CT(0), CT(0), CT(0)};
      bool hit = false;
      if (c < Mt) {
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (S.seg[lo + step] <= c) lo += step;
        const int tl = lo;
        hit = Pol::mesh_contact(p, mesh, lb, w0 + tl, (int)(c - S.seg[tl]), P[w0 + tl],
                                V[w0 + tl], W[w0 + tl], stamp_now, stamp_new, c6);
        if (hit) ++nmesh;
      }
      const unsigned hm = __ballot_sync(full, hit);
#pragma unroll
      for (int k = 0; k < 6; ++k) S.contrib[lane][k] = c6[k];
      __syncwarp();
      const uint32_t a = my_a > c0 ? my_a : c0;
      const uint32_t b = my_b < c0 + 32 ? my_b : c0 + 32;
      for (uint32_t jj = a; jj < b; ++jj)
        if (hm >> (jj - c0) & 1u) acc.add(S.contrib[jj - c0]);
      __syncwarp();
    }
  }

  // C: integration of the lane's own particle
  bool disp = false, bad = false;
  if (valid)
    Pol::finish(p, sb, ph, lb, mesh, t, (meta >> 16) & 0xffu, false, P[t], V[t],
                W[t], acc, stamp_now, stamp_new, forces, nmesh, disp, bad);

  count_and_flag(ctl, npair, nmesh, disp, bad);
}

template <typename Pol>
void launch_step_warp(cudaStream_t st, Ctl* ctl, const Params& p, StateBufs sb, Lists L,
                      MeshDev mesh, double* forces) {
  if (p.step_warps == 8)
    k_step_warp<Pol, 8><<<(unsigned)((p.n + 255) / 256), 256, 0, st>>>(ctl, p, sb, L, mesh,
                                                                        forces);
  else
    k_step_warp<Pol, 4><<<(unsigned)((p.n + 127) / 128), 128, 0, st>>>(ctl, p, sb, L, mesh,
                                                                        forces);
}

}  // namespace dem
