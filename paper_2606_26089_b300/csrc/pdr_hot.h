// Host-side construction of the shared-memory card cache (HotCard) from an
// expanded DevCard.  Writes into caller storage; allocates nothing.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>

#include "pdr_internal.h"

namespace pdr {

// Returns the number of bytes written (a multiple of 16), or 0 if the card's
// tables do not fit in cap bytes (or PDR_HOT_MAX_BYTES).
inline size_t build_hot_card(const DevCard& D, unsigned char* out, size_t cap) {
  if (cap > PDR_HOT_MAX_BYTES) cap = PDR_HOT_MAX_BYTES;
  if (cap < sizeof(HotCard)) return 0;
  HotCard& H = *reinterpret_cast<HotCard*>(out);
  std::memset(&H, 0, sizeof H);
  float* data = reinterpret_cast<float*>(out + sizeof(HotCard));
  const size_t max_floats = (cap - sizeof(HotCard)) / sizeof(float);
  size_t nf = 0;
  auto need = [&](size_t k) { return nf + k <= max_floats; };
  for (int calo = 0; calo < 2; ++calo) {
    const DevCalo& C = D.calo[calo];
    HotCalo& hc = H.calo[calo];
    hc.nring = C.nring;
    hc.m = C.nring / 2;
    hc.nseg = C.nseg;
    if (!need((size_t)C.nring + 1)) return 0;
    hc.edge_off = (int32_t)nf;
    for (int j = 0; j <= C.nring; ++j) data[nf++] = C.edge[j];
    for (int s = 0; s < C.nseg; ++s) {
      HotSeg& hs = hc.seg[s];
      hs.lo = C.seg_lo[s];
      hs.hi = C.seg_hi[s];
      hs.scale = C.seg_scale[s];
      hs.n = C.seg_n[s];
      hs.first = C.seg_first[s];
      const int r_pos = hc.m + hs.first;           // lowest ring of the segment, eta > 0
      const int r_neg = hc.m - hs.first - hs.n;    // lowest ring of the segment, eta < 0
      hs.nphi = C.nphi[r_pos];
      hs.base_pos = C.base[r_pos];
      hs.base_neg = C.base[r_neg];
      hs.phi_scale = C.phi_scale[r_pos];
      if (!need(2 * (size_t)hs.nphi + 1)) return 0;
      hs.phioff = (int32_t)nf;
      const float* src = D.phi_pool + C.phioff[r_pos];
      for (int k = 0; k < 2 * hs.nphi + 1; ++k) data[nf++] = src[k];
    }
    // per ring, 16-byte aligned: eta_c, 1 / cosh(eta_c), first tower id, and
    // phi-table offset | nphi << 16 | resolution row << 27
    while (nf & 3) {
      if (!need(1)) return 0;
      data[nf++] = 0.0f;
    }
    if (!need(4 * (size_t)C.nring)) return 0;
    hc.ring_off = (int32_t)nf;
    for (int r = 0; r < C.nring; ++r) {
      const int jj = r >= hc.m ? r - hc.m : hc.m - 1 - r;
      int s = 0;
      while (s < C.nseg - 1 && jj >= hc.seg[s].first + hc.seg[s].n) ++s;
      const uint32_t phioff = (uint32_t)hc.seg[s].phioff, nphi = (uint32_t)C.nphi[r], rb = (uint32_t)C.resbin[r];
      if (phioff >= (1u << 16) || nphi >= (1u << 11) || rb >= (1u << 5)) return 0;
      const uint32_t packed = phioff | (nphi << 16) | (rb << 27);
      const int32_t base = C.base[r];
      data[nf++] = C.eta_c[r];
      data[nf++] = C.inv_cosh_c[r];
      std::memcpy(&data[nf++], &base, sizeof(float));
      std::memcpy(&data[nf++], &packed, sizeof(float));
    }
  }
  H.R = D.R; H.L = D.L; H.kB = D.kB; H.L_lo = D.L_lo; H.kB_lo = D.kB_lo;
  H.Bsign = D.Bsign; H.has_field = D.has_field;
  H.trk_npt = D.trk_npt; H.trk_neta = D.trk_neta; H.id_n = D.id_n;
  for (int k = 0; k < 4; ++k) H.res_n[k] = D.res_n[k];
  std::memcpy(H.trk_pt_edges, D.trk_pt_edges, sizeof H.trk_pt_edges);
  std::memcpy(H.trk_eta_edges, D.trk_eta_edges, sizeof H.trk_eta_edges);
  std::memcpy(H.id_edges, D.id_edges, sizeof H.id_edges);
  std::memcpy(H.res_edges, D.res_edges, sizeof H.res_edges);
  for (int c = 0; c < 4; ++c)
    for (int k = 0; k < PDR_MAXEDGE; ++k)
      H.res[c][k] = make_float4(D.res_a2[c][k], D.res_b2[c][k], D.res_c2[c][k], D.res_d2[c][k]);
  std::memcpy(H.cR_hi, D.cR_hi, sizeof H.cR_hi);
  std::memcpy(H.cR_lo, D.cR_lo, sizeof H.cR_lo);
  std::memcpy(H.trk_T, D.trk_T, sizeof H.trk_T);
  std::memcpy(H.id_T, D.id_T, sizeof H.id_T);
  std::memcpy(H.e_min, D.e_min, sizeof H.e_min);
  std::memcpy(H.s_min, D.s_min, sizeof H.s_min);
  H.cand_ptmin = D.cand_ptmin; H.dr2max = D.dr2max; H.dr2min = D.dr2min;
  H.iso_ptmin = D.iso_ptmin; H.imax = D.imax;
  {
    // (a cone radius that is not a finite number puts every object in one bin)
    const double dr = std::sqrt((double)D.dr2max);
    if (std::isfinite(dr)) {
      const double w = std::max(1.001 * dr, 16.0 / PDR_ISO_BINS);
      H.iso_inv_w = (float)(1.0 / w);
      H.iso_nbin = std::max(1, std::min(PDR_ISO_BINS, (int)std::ceil(16.0 / w)));
    } else {
      H.iso_inv_w = 0.0f;
      H.iso_nbin = 1;
    }
  }
  const size_t used = nf;
  nf = (nf + 3) & ~size_t(3);  // 16-byte multiple
  if (nf > max_floats) return 0;
  for (size_t k = used; k < nf; ++k) data[k] = 0.0f;
  H.data_floats = (int32_t)nf;
  return sizeof(HotCard) + nf * sizeof(float);
}

}  // namespace pdr
