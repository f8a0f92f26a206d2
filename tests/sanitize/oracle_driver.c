/* Runs the oracle's entry points over a batch read from a file, for the
 * AddressSanitizer / UndefinedBehaviorSanitizer build of the tests (test
 * infrastructure: memory-safety evidence for the oracle).
 *
 * File: magic "PDRS", u64 n_events, u64 n_particles, u32 has_vz, the card
 * (oracle_card bytes), u64 offsets[n_events + 1], f32 pt, eta, phi, mass,
 * i32 pdg, i8 charge, f32 vz (if has_vz).  Exit status 0 when every call
 * returned normally. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static void* take(FILE* f, size_t n) {
  void* p = malloc(n ? n : 1);
  if (!p || (n && fread(p, 1, n, f) != n)) {
    fprintf(stderr, "short file\n");
    exit(2);
  }
  return p;
}

int main(int argc, char** argv) {
  if (argc != 2) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  char magic[4];
  uint64_t ne, np;
  uint32_t has_vz;
  if (fread(magic, 1, 4, f) != 4 || memcmp(magic, "PDRS", 4) || fread(&ne, 8, 1, f) != 1 ||
      fread(&np, 8, 1, f) != 1 || fread(&has_vz, 4, 1, f) != 1)
    return 2;
  oracle_card* card = (oracle_card*)take(f, sizeof(oracle_card));
  uint64_t* off = (uint64_t*)take(f, 8 * (ne + 1));
  float* pt = (float*)take(f, 4 * np);
  float* eta = (float*)take(f, 4 * np);
  float* phi = (float*)take(f, 4 * np);
  float* mass = (float*)take(f, 4 * np);
  int32_t* pdg = (int32_t*)take(f, 4 * np);
  int8_t* charge = (int8_t*)take(f, np);
  float* vz = has_vz ? (float*)take(f, 4 * np) : NULL;
  fclose(f);

  long n_records = 0;
  for (uint64_t e = 0; e < ne; ++e) {
    const int64_t a = (int64_t)off[e], n = (int64_t)(off[e + 1] - off[e]);
    const size_t cap = n > 0 ? (size_t)n : 1;
    or_particle* part = (or_particle*)calloc(cap, sizeof *part);
    or_track* trk = (or_track*)calloc(cap, sizeof *trk);
    or_tower* twr = (or_tower*)calloc(cap, sizeof *twr);
    or_cand* cand = (or_cand*)calloc(cap, sizeof *cand);
    const int32_t mcap = 64 + 16 * (int32_t)n;
    or_marginal* marg = (or_marginal*)calloc((size_t)mcap, sizeof *marg);
    or_counts cnt;
    int rc = oracle_run_event(card, n, pt + a, eta + a, phi + a, mass + a, pdg + a, charge + a,
                              vz ? vz + a : NULL, 7, (uint32_t)e, 1e-5, NULL, 0, part, trk, twr, cand, marg,
                              mcap, &cnt);
    if (rc) { fprintf(stderr, "run_event %d\n", rc); return 1; }
    n_records += cnt.n_trk + cnt.n_twr + cnt.n_cand;
    /* the response's marginal decisions, each flipped once, must be accepted */
    for (int32_t k = 0; k < cnt.n_marg && k < mcap && k < 3; ++k) {
      or_flip fl = {marg[k].kind, marg[k].id, marg[k].aux, marg[k].aux2};
      or_counts c2;
      rc = oracle_run_event(card, n, pt + a, eta + a, phi + a, mass + a, pdg + a, charge + a,
                            vz ? vz + a : NULL, 7, (uint32_t)e, 1e-5, &fl, 1, part, trk, twr, cand, marg,
                            mcap, &c2);
      if (rc) { fprintf(stderr, "flip %d\n", rc); return 1; }
    }
    /* clustering of the generated particles, all three pp algorithms and e+e- */
    double* px = (double*)malloc(cap * sizeof(double));
    double* py = (double*)malloc(cap * sizeof(double));
    double* pz = (double*)malloc(cap * sizeof(double));
    double* en = (double*)malloc(cap * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
      const double p_t = pt[a + i], h = eta[a + i], ph = phi[a + i];
      px[i] = p_t * cos(ph); py[i] = p_t * sin(ph); pz[i] = p_t * sinh(h);
      en[i] = sqrt(px[i] * px[i] + py[i] * py[i] + pz[i] * pz[i] + (double)mass[a + i] * mass[a + i]);
    }
    or_jet* jets = (or_jet*)calloc(cap, sizeof *jets);
    int32_t* msteps = (int32_t*)calloc(cap, sizeof(int32_t));
    for (int alg = -1; alg <= 2 && n <= 400; ++alg) {  /* (the oracle's clustering is cubic in n) */
      int32_t nm = 0;
      const int ee = alg == 2;
      const int32_t nj = oracle_cluster_forced(n, px, py, pz, en, ee ? 1.0 : alg, ee ? 0.7 : 0.5, 5.0, 1, ee, jets,
                                               &nm, NULL, 0, msteps, (int32_t)cap);
      if (nj < 0) { fprintf(stderr, "cluster %d\n", nj); return 1; }
      if (nm > 0) {  /* force the first marginal step */
        int32_t nm2 = 0;
        const int32_t s = msteps[0];
        if (oracle_cluster_forced(n, px, py, pz, en, ee ? 1.0 : alg, ee ? 0.7 : 0.5, 5.0, 1, ee, jets, &nm2, &s, 1,
                                  NULL, 0) < 0) {
          fprintf(stderr, "forced cluster\n");
          return 1;
        }
      }
    }
    /* impact parameters of every charged particle, vertices displaced */
    oracle_ip_params ip = {10e-6, 50e-6, 30e-6, 80e-6};
    for (int64_t i = 0; i < n; ++i) {
      if (!charge[a + i]) continue;
      double out[4];
      oracle_track_ip_smeared(card, &ip, pt[a + i], eta[a + i], phi[a + i], charge[a + i], 1e-3 * (double)(i % 7),
                              -2e-3 * (double)(i % 5), vz ? vz[a + i] : 0.0, 7, (uint32_t)e, (uint32_t)i, out);
    }
    free(px); free(py); free(pz); free(en); free(jets); free(msteps);
    free(part); free(trk); free(twr); free(cand); free(marg);
  }
  /* the threaded batch form */
  uint32_t* counts = (uint32_t*)calloc(ne ? ne : 1, 4 * sizeof(uint32_t));
  if (oracle_run_batch(card, (int64_t)ne, off, pt, eta, phi, mass, pdg, charge, vz, 7, 0, 3, counts)) return 1;
  /* pile-up draws with forced truncation decisions */
  oracle_pileup pu = {30.0, 0.05, 0.02, 160e-12, 100e-12, 1, 0};
  uint64_t T[4096];
  const int32_t K = oracle_poisson_thresholds(pu.mean, T, 4096);
  if (K <= 0) return 1;
  for (uint32_t e = 0; e < 40; ++e) {
    int32_t nn;
    uint32_t idx[512], mo[3 * 64];
    double z[512], t[512], zh, th;
    const int32_t m = oracle_pileup_draws_forced(&pu, T, K, 1000, 7, e, 1e-2, &nn, idx, z, t, 512, &zh, &th, NULL, 0,
                                                 mo, 64);
    if (m < 0) return 1;
    if (m > 0) {
      int32_t nn2;
      (void)oracle_pileup_draws_forced(&pu, T, K, 1000, 7, e, 1e-2, &nn2, idx, z, t, 512, &zh, &th, mo, 1, NULL, 0);
    }
  }
  printf("ok %llu events, %ld records\n", (unsigned long long)ne, n_records);
  free(counts); free(card); free(off); free(pt); free(eta); free(phi); free(mass); free(pdg); free(charge); free(vz);
  return 0;
}
