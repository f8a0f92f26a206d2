// Detector-card expansion (host side): the raw card of include/pdr.h into the
// device tables (DevCard).  Fixed-size storage only (no heap), so both the
// context path (pdr_card_load) and the allocation-free entry point use this one
// definition of edges, tower numbering and thresholds.
//
// Readings (the paper gives no binning formulas; App. D.1 only names the
// per-module card parameters): ring edges inside an eta segment are
// lo + ((hi - lo) k) / n in double with the segment ends exact, mirrored at
// eta = 0; phi edges are -pi + (2 pi k) / n_phi; decisions are taken on the
// float32 edges; efficiency thresholds are floor(eff 2^32) (eff = 1: 2^32).
#pragma once

#include <cmath>
#include <cstring>

#include "pdr_internal.h"

namespace pdr {

int set_last_error(int code, const char* msg);

inline unsigned long long eff_threshold(double eff) {
  if (eff >= 1.0) return 4294967296ull;
  if (!(eff > 0.0)) return 0ull;
  return (unsigned long long)std::floor(eff * 4294967296.0);
}

// Strictly increasing in float32 (the precision decisions are taken in).
inline bool increasing_f32(const double* v, int n) {
  for (int i = 0; i + 1 < n; ++i)
    if (!((float)v[i] < (float)v[i + 1])) return false;
  return true;
}

inline int expand_calo(const pdr_card* c, int calo, DevCalo& D, float* pool, int& pool_used) {
  const int nseg = c->nseg[calo];
  if (nseg < 1 || nseg > PDR_MAXSEG) return set_last_error(PDR_ECARD, "calorimeter needs 1..4 eta segments");
  double p[PDR_MAXRING / 2 + 1];
  int pn[PDR_MAXRING / 2];
  int m = 0;
  double lo = 0.0;
  p[0] = 0.0;
  std::memset(&D, 0, sizeof D);
  D.nseg = nseg;
  for (int s = 0; s < nseg; ++s) {
    const double hi = c->seg_eta_hi[calo][s];
    const int n = c->seg_neta[calo][s];
    const int nphi = c->seg_nphi[calo][s];
    if (!(hi > lo) || n < 1 || nphi < 1 || nphi > PDR_MAXPHI)
      return set_last_error(PDR_ECARD, "bad calorimeter segment (eta_hi must increase, n_eta >= 1, 1 <= n_phi <= 1024)");
    if (m + n > PDR_MAXRING / 2) return set_last_error(PDR_ECARD, "too many eta rings (max 512)");
    D.seg_lo[s] = (float)lo;
    D.seg_hi[s] = (float)hi;
    D.seg_scale[s] = (float)(n / (hi - lo));
    D.seg_n[s] = n;
    D.seg_first[s] = m;
    for (int k = 1; k <= n; ++k) {
      p[m + k] = (k == n) ? hi : lo + ((hi - lo) * (double)k) / (double)n;
      pn[m + k - 1] = nphi;
    }
    m += n;
    lo = hi;
  }
  D.nring = 2 * m;
  double edge[PDR_MAXRING + 1];
  int nphi[PDR_MAXRING];
  for (int j = 0; j <= m; ++j) {
    edge[m + j] = p[j];
    edge[m - j] = -p[j];
  }
  edge[m] = 0.0;
  for (int r = 0; r < m; ++r) {
    nphi[m + r] = pn[r];
    nphi[m - 1 - r] = pn[r];
  }
  for (int j = 0; j <= 2 * m; ++j) D.edge[j] = (float)edge[j];
  for (int j = 0; j < 2 * m; ++j)
    if (!(D.edge[j] < D.edge[j + 1])) return set_last_error(PDR_ECARD, "eta ring edges not increasing in float32");
  // phi tables are shared by the rings of a calorimeter with the same bin count
  int tab_np[2 * PDR_MAXSEG], tab_off[2 * PDR_MAXSEG], ntab = 0;
  int base = 0;
  for (int r = 0; r < 2 * m; ++r) {
    D.base[r] = base;
    D.nphi[r] = nphi[r];
    base += nphi[r];
    int off = -1;
    for (int t = 0; t < ntab; ++t)
      if (tab_np[t] == nphi[r]) off = tab_off[t];
    if (off < 0) {
      const int np = nphi[r];
      if (pool_used + 2 * np + 1 > PDR_PHIPOOL || ntab >= 2 * PDR_MAXSEG)
        return set_last_error(PDR_ECARD, "phi table pool exhausted");
      off = pool_used;
      for (int k = 0; k <= np; ++k)
        pool[off + k] = (float)(k == 0 ? -M_PI : (k == np ? M_PI : -M_PI + (2.0 * M_PI * (double)k) / (double)np));
      for (int k = 0; k < np; ++k) {
        const double e0 = k == 0 ? -M_PI : -M_PI + (2.0 * M_PI * (double)k) / (double)np;
        const double e1 = k + 1 == np ? M_PI : -M_PI + (2.0 * M_PI * (double)(k + 1)) / (double)np;
        pool[off + np + 1 + k] = (float)(0.5 * (e0 + e1));
      }
      pool_used += 2 * np + 1;
      tab_np[ntab] = np;
      tab_off[ntab] = off;
      ++ntab;
    }
    D.phioff[r] = off;
    D.phi_scale[r] = (float)(nphi[r] / (2.0 * M_PI));
    const double ec = 0.5 * (edge[r] + edge[r + 1]);
    D.eta_c[r] = (float)ec;
    D.inv_cosh_c[r] = (float)(1.0 / std::cosh(ec));
  }
  D.ntowers = base;
  // ring groups in ring order: negative-side segments outermost first, then
  // positive-side segments innermost first
  D.ngroup = 2 * nseg;
  for (int s = 0; s < nseg; ++s) {
    const int gn = nseg - 1 - s, gp = nseg + s;
    D.grp_first[gn] = m - D.seg_first[s] - D.seg_n[s];
    D.grp_first[gp] = m + D.seg_first[s];
    D.grp_nphi[gn] = D.grp_nphi[gp] = c->seg_nphi[calo][s];
    D.grp_base[gn] = D.base[D.grp_first[gn]];
    D.grp_base[gp] = D.base[D.grp_first[gp]];
  }
  if (base >= (1 << 24)) return set_last_error(PDR_ECARD, "too many towers (max 2^24 per calorimeter)");
  return PDR_OK;
}

// Validates the card (positive R and L, finite B, table sizes, increasing
// edges, efficiencies in [0, 1], non-negative resolution terms) and expands it.
inline int expand_card(const pdr_card* c, DevCard& D) {
  std::memset(&D, 0, sizeof D);
  if (!(c->R > 0.0) || !(c->L > 0.0) || !std::isfinite(c->B))
    return set_last_error(PDR_ECARD, "need R > 0, L > 0, finite B");
  int pool_used = 0;
  for (int calo = 0; calo < 2; ++calo) {
    int rc = expand_calo(c, calo, D.calo[calo], D.phi_pool, pool_used);
    if (rc) return rc;
  }
  D.R = (float)c->R;
  D.L = (float)c->L;
  D.L_lo = (float)(c->L - (double)D.L);
  const double kB = 0.299792458 * std::fabs(c->B);
  D.kB = (float)kB;
  D.kB_lo = (float)(kB - (double)D.kB);
  D.Bsign = c->B > 0.0 ? 1 : -1;
  D.has_field = c->B != 0.0;
  for (int q = 1; q <= PDR_MAXQ; ++q) {
    const double cR = 0.299792458 * std::fabs((double)q) * std::fabs(c->B) * c->R;
    D.cR_hi[q] = (float)cR;
    D.cR_lo[q] = (float)(cR - (double)D.cR_hi[q]);
  }
  // efficiencies
  if (c->trk_npt < 1 || c->trk_npt > PDR_MAXEDGE || c->trk_neta < 1 || c->trk_neta > PDR_MAXEDGE ||
      c->id_n < 1 || c->id_n > PDR_MAXEDGE)
    return set_last_error(PDR_ECARD, "efficiency tables need 1..8 edges per axis");
  if (!increasing_f32(c->trk_pt_edges, c->trk_npt) || !increasing_f32(c->trk_eta_edges, c->trk_neta) ||
      !increasing_f32(c->id_edges, c->id_n))
    return set_last_error(PDR_ECARD, "efficiency table edges must increase");
  D.trk_npt = c->trk_npt;
  D.trk_neta = c->trk_neta;
  for (int k = 0; k < PDR_MAXEDGE; ++k) {
    D.trk_pt_edges[k] = D.trk_eta_edges[k] = D.id_edges[k] = INFINITY;
    for (int comp = 0; comp < 4; ++comp) D.res_edges[comp][k] = INFINITY;
  }
  for (int k = 0; k < c->trk_npt; ++k) D.trk_pt_edges[k] = (float)c->trk_pt_edges[k];
  for (int k = 0; k < c->trk_neta; ++k) D.trk_eta_edges[k] = (float)c->trk_eta_edges[k];
  for (int t = 0; t < 3; ++t)
    for (int i = 0; i < c->trk_npt; ++i)
      for (int j = 0; j < c->trk_neta; ++j) {
        const double e = c->trk_eff[t][i][j];
        if (!(e >= 0.0 && e <= 1.0)) return set_last_error(PDR_ECARD, "tracking efficiency outside [0, 1]");
        D.trk_T[t][i][j] = eff_threshold(e);
      }
  D.id_n = c->id_n;
  for (int k = 0; k < c->id_n; ++k) D.id_edges[k] = (float)c->id_edges[k];
  for (int t = 0; t < 3; ++t)
    for (int k = 0; k < c->id_n; ++k) {
      const double e = c->id_eff[t][k];
      if (!(e >= 0.0 && e <= 1.0)) return set_last_error(PDR_ECARD, "identification efficiency outside [0, 1]");
      D.id_T[t][k] = eff_threshold(e);
    }
  // resolutions
  for (int comp = 0; comp < 4; ++comp) {
    const int n = c->res_n[comp];
    if (n < 1 || n > PDR_MAXEDGE || !increasing_f32(c->res_edges[comp], n))
      return set_last_error(PDR_ECARD, "resolution tables need 1..8 increasing |eta| edges");
    D.res_n[comp] = n;
    for (int k = 0; k < n; ++k) {
      D.res_edges[comp][k] = (float)c->res_edges[comp][k];
      const double a = c->res_abcd[comp][k][0], b = c->res_abcd[comp][k][1];
      const double cc = c->res_abcd[comp][k][2], d = c->res_abcd[comp][k][3];
      if (!(a >= 0 && b >= 0 && cc >= 0 && d >= 0)) return set_last_error(PDR_ECARD, "negative resolution coefficient");
      D.res_a2[comp][k] = (float)(a * a);
      D.res_b2[comp][k] = (float)(b * b);
      D.res_c2[comp][k] = (float)(cc * cc);
      D.res_d2[comp][k] = (float)(d * d);
    }
  }
  // tower resolution row of each ring: the |eta| bin of its centre
  for (int calo = 0; calo < 2; ++calo) {
    DevCalo& C = D.calo[calo];
    const int comp = calo == 0 ? RES_ECAL : RES_HCAL;
    for (int r = 0; r < C.nring; ++r) {
      int k = -1;
      for (int j = 0; j < c->res_n[comp]; ++j)
        if ((float)c->res_edges[comp][j] <= std::fabs(C.eta_c[r])) k = j;
      C.resbin[r] = k < 0 ? 0 : k;
    }
    D.e_min[calo] = (float)c->e_min[calo];
    D.s_min[calo] = (float)c->s_min[calo];
  }
  D.cand_ptmin = (float)c->cand_ptmin;
  D.dr2max = (float)(c->iso_dr * c->iso_dr);
  D.dr2min = (float)(c->iso_drmin * c->iso_drmin);
  D.iso_ptmin = (float)c->iso_ptmin;
  D.imax = (float)c->iso_imax;
  return PDR_OK;
}

}  // namespace pdr
