// One evaluation per pair (Sec. 3.2 evaluates each pair once and applies the
// result to both particles).  A pair kernel runs the contact law once per
// touching pair, at the entry of its lower-caller-index particle i whose
// partner index is above i's (an "upper" entry), writes the force on i and
// the torques on i and j to that entry's result record, and marks the pair in
// both particles' touch masks (bit k = list entry k touched this step;
// integer atomics only).  A gather kernel then walks, for every particle, the
// set bits of its mask in ascending order -- ascending partner caller index --
// and adds each contribution: an upper entry's force and torque on i, or, for
// a lower entry, the partner's record found through the mirror index (force
// negated, torque on j).  These are the values and the order of evaluating
// the pair from both sides.  Then mesh contacts and integration follow as in
// the one-kernel step, and the gather clears the mask for the next step.
// Friction history lives at the upper entries only.  DEM_FP64, bound by the
// FP64 pipe, runs this way.  For DEM_MIXED (latency bound) it was measured
// slower than the one-kernel scheme of dem_step_warp.cuh: on the 400k drum
// the pair and gather kernels took 75.9 + 49.4 us against 108.4 us, since
// halving the entries and laws per warp does not halve a warp's chain of
// dependent loads, and the state is read twice.
#pragma once

#include "dem_internal.cuh"
#include "dem_law.cuh"
#include "dem_math.cuh"
#include "dem_step_common.cuh"
#include "dem_step_warp.cuh"

namespace dem {

// A pair's result in canonical orientation: force on i, torques on i and j.
template <typename T>
struct PairOut;
template <>
struct PairOut<double> {  // 80 bytes
  double f[3], ti[3], tj[3], pad;
};
template <>
struct __align__(16) PairOut<float> {  // 48 bytes
  float f[3], ti[3], tj[3], pad[3];
};

__device__ __forceinline__ void put_out(PairOut<float>* r, const LawOut<float>& o) {
  PairOut<float> a;
  a.f[0] = o.f.x; a.f[1] = o.f.y; a.f[2] = o.f.z;
  a.ti[0] = o.ti.x; a.ti[1] = o.ti.y; a.ti[2] = o.ti.z;
  a.tj[0] = o.tj.x; a.tj[1] = o.tj.y; a.tj[2] = o.tj.z;
  a.pad[0] = a.pad[1] = a.pad[2] = 0.f;
  *r = a;
}

__device__ __forceinline__ void put_out(PairOut<double>* r, const LawOut<double>& o) {
  PairOut<double> a;
  a.f[0] = o.f.x; a.f[1] = o.f.y; a.f[2] = o.f.z;
  a.ti[0] = o.ti.x; a.ti[1] = o.ti.y; a.ti[2] = o.ti.z;
  a.tj[0] = o.tj.x; a.tj[1] = o.tj.y; a.tj[2] = o.tj.z;
  a.pad = 0.0;
  *r = a;
}
// contribution to i (an upper entry) or to j (a lower entry)
template <typename T>
__device__ __forceinline__ void get_out(const PairOut<T>* r, bool on_i, T c6[6]) {
  const T* t = on_i ? r->ti : r->tj;
  if (on_i) {
    c6[0] = r->f[0]; c6[1] = r->f[1]; c6[2] = r->f[2];
  } else {
    c6[0] = -r->f[0]; c6[1] = -r->f[1]; c6[2] = -r->f[2];
  }
  c6[3] = t[0]; c6[4] = t[1]; c6[5] = t[2];
}

constexpr int kPairWarps = 4;

// Phases A and B of the warp kernel (dem_step_warp.cuh) over the warp's
// upper entries only: a cheap overlap pre-test queues the candidates, then
// the law runs for 32 queued pairs at a time.
template <typename Pol, int MinBlocks>
__global__ void __launch_bounds__(32 * kPairWarps, MinBlocks)
k_pairs(Ctl* ctl, Params p, StateBufs sb, Lists L, PairOut<typename Pol::T>* res,
        unsigned long long* touch) {
  using Rec = typename Pol::Rec;
  using Hist = typename Pol::Hist;
  using CT = typename Pol::T;
  __shared__ uint32_t seg_s[kPairWarps][33];
  __shared__ uint32_t off_s[kPairWarps][32];
  __shared__ uint32_t qent_s[kPairWarps][kQueueMax];
  __shared__ uint32_t qslot_s[kPairWarps][kQueueMax];
  __shared__ uint8_t qlane_s[kPairWarps][kQueueMax];
  __shared__ uint8_t qk_s[kPairWarps][kQueueMax];
  __shared__ uint8_t nlow_s[kPairWarps][32];
  if (ctl->status) return;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* seg = seg_s[wib];
  uint32_t* offw = off_s[wib];
  uint32_t* qent = qent_s[wib];
  uint32_t* qslot = qslot_s[wib];
  uint8_t* qlane = qlane_s[wib];
  uint8_t* qk = qk_s[wib];
  uint8_t* nlw = nlow_s[wib];
  const int n = p.n;
  const int w0 = (blockIdx.x * kPairWarps + wib) * 32;
  const int t = w0 + lane;
  const bool valid = t < n;
  const uint32_t ph = ctl->phase & 1u, lph = ctl->lphase & 1u;
  const uint32_t stamp_now = (uint32_t)ctl->step, stamp_new = stamp_now + 1u;
  const Rec* P = static_cast<const Rec*>(buf_of(sb.P, ph));
  const Rec* V = static_cast<const Rec*>(buf_of(sb.V, ph));
  const Rec* W = static_cast<const Rec*>(buf_of(sb.W, ph));
  const ListBuf lb = list_of(L, lph);
  Hist* Hh = static_cast<Hist*>(lb.hpp);
  const uint32_t meta = valid ? lb.meta[t] : 0u;
  const uint32_t nn = meta & 0xffu, nlow = (meta >> 8) & 0xffu;
  const uint32_t incl = warp_incl_scan(nn - nlow);
  seg[lane + 1] = incl;
  if (lane == 0) seg[0] = 0;
  // offw: the lane's first upper entry; the entry's list index is nlow + local
  offw[lane] = valid ? lb.offs[t] + nlow : 0u;
  nlw[lane] = (uint8_t)nlow;
  const uint32_t Eu = __shfl_sync(full, incl, 31);
  __syncwarp();
  uint32_t npair = 0;
  uint32_t e0 = 0;
  while (e0 < Eu) {
    // A: pre-test, queue the candidates (entry, partner slot, owner lane, list index)
    uint32_t qn = 0;
    for (; e0 < Eu && qn + 32 <= (uint32_t)kQueueMax; e0 += 32) {
      const uint32_t e = e0 + lane;
      bool hit = false;
      uint32_t ent = 0, u = 0, k = 0;
      int tl = 0;
      if (e < Eu) {
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (seg[lo + step] <= e) lo += step;
        tl = lo;
        const uint32_t local = e - seg[tl];
        ent = offw[tl] + local;
        k = nlw[tl] + local;
        u = lb.nbr[ent];
        hit = Pol::near(P[w0 + tl], P[u]);
      }
      const unsigned m = __ballot_sync(full, hit);
      if (hit) {
        const uint32_t pos = qn + __popc(m & ((1u << lane) - 1u));
        qent[pos] = ent;
        qslot[pos] = u;
        qlane[pos] = (uint8_t)tl;
        qk[pos] = (uint8_t)k;
      }
      qn += __popc(m);
    }
    __syncwarp();
    // B: the law for 32 queued pairs at a time, results to their entries
    for (uint32_t i0 = 0; i0 < qn; i0 += 32) {
      const uint32_t i = i0 + lane;
      if (i < qn) {
        const uint32_t ent = qent[i], u = qslot[i];
        const int tl = qlane[i];
        Hist h = Hh[ent];
        LawOut<CT> o;
        if (Pol::pair_law(p, P[w0 + tl], P[u], V[w0 + tl], V[u], W[w0 + tl], W[u],
                          Pol::aux(lb, w0 + tl), Pol::aux(lb, u), h, stamp_now, stamp_new, o)) {
          Hh[ent] = h;
          put_out(res + ent, o);
          atomicOr(&touch[w0 + tl], 1ull << qk[i]);
          atomicOr(&touch[u], 1ull << lb.back[ent]);
          npair += 2;  // two directed entries, as the stats count them
        }
      }
    }
    __syncwarp();
  }
  count_and_flag(ctl, npair, 0u, false, false);
}

// Per particle: the pair sums over the touched entries in list order, then
// mesh contacts and integration; the touch mask is cleared for the next step.
template <typename Pol, int MinBlocks>
__global__ void __launch_bounds__(128, MinBlocks)
k_gather(Ctl* ctl, Params p, StateBufs sb, Lists L, MeshDev mesh,
         const PairOut<typename Pol::T>* res, unsigned long long* touch, double* forces) {
  using Rec = typename Pol::Rec;
  using CT = typename Pol::T;
  if (ctl->status) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = t < p.n;
  const uint32_t ph = ctl->phase & 1u, lph = ctl->lphase & 1u;
  const uint32_t stamp_now = (uint32_t)ctl->step, stamp_new = stamp_now + 1u;
  const ListBuf lb = list_of(L, lph);
  uint32_t nmesh = 0;
  bool disp = false, bad = false;
  if (valid) {
    const Rec* P = static_cast<const Rec*>(buf_of(sb.P, ph));
    const Rec* V = static_cast<const Rec*>(buf_of(sb.V, ph));
    const Rec* W = static_cast<const Rec*>(buf_of(sb.W, ph));
    const uint32_t meta = lb.meta[t];
    const uint32_t nlow = (meta >> 8) & 0xffu;
    const uint32_t off = lb.offs[t];
    unsigned long long m = touch[t];
    if (m) touch[t] = 0ull;
    typename Pol::Acc acc;
    acc.zero();
    CT c6[6];
    while (m) {
      const uint32_t k = (uint32_t)(__ffsll((long long)m) - 1);
      m &= m - 1ull;
      const bool lower = k < nlow;
      const uint32_t e = lower ? lb.mir[off + k] : off + k;
      get_out(res + e, !lower, c6);
      acc.add(c6);
    }
    Pol::finish(p, sb, ph, lb, mesh, t, (meta >> 16) & 0xffu, true, P[t], V[t], W[t], acc,
                stamp_now, stamp_new, forces, nmesh, disp, bad);
  }
  count_and_flag(ctl, 0u, nmesh, disp, bad);
}

template <typename Pol, int PairMinBlocks, int GatherMinBlocks>
void launch_step_pairs(cudaStream_t st, Ctl* ctl, const Params& p, StateBufs sb, Lists L,
                       MeshDev mesh, double* forces) {
  using Out = PairOut<typename Pol::T>;
  Out* res = static_cast<Out*>(p.pair_res);
  k_pairs<Pol, PairMinBlocks>
      <<<(unsigned)((p.n + 32 * kPairWarps - 1) / (32 * kPairWarps)), 32 * kPairWarps, 0, st>>>(
          ctl, p, sb, L, res, p.pair_touch);
  k_gather<Pol, GatherMinBlocks><<<(unsigned)((p.n + 127) / 128), 128, 0, st>>>(
      ctl, p, sb, L, mesh, res, p.pair_touch, forces);
}

}  // namespace dem
