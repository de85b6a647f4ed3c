// layout_probe.cu -- test infrastructure: checks on the host that the
// per-instance shared-memory layouts of the solver (make_lay, make_reg_lay,
// make_ks_lay, make_adj) hold every region the kernels index, for every node count,
// control size and CTA size the library accepts, and the index algebra of
// PIPG form 3's butterfly exchanges.  Built by
// tests/test_layout.py once per model; prints "OK <cases>" or the failures.
#include <cstdio>

#include "pdg_adjoint.cuh"

using namespace pdg;

static int bad = 0;
#define CHECK(cond, N, nu, T)                                                                     \
  do {                                                                                            \
    if (!(cond)) {                                                                                \
      if (bad < 20) std::printf("FAIL N=%d nu=%d T=%d: %s\n", (N), (nu), (T), #cond);            \
      ++bad;                                                                                      \
    }                                                                                             \
  } while (0)

// PIPG form 3's butterflies, lane by lane on the host: with every lane's
// partial sums stored in the order of ks_perm, rounds that keep the first
// half of the stored entries and add the partner's second half (as
// ks_rs_round does) leave lane sel the full sums of entries (n / M) sel ..
// (n / M) sel + n / M - 1, and the inverse rounds (ks_ag_round) return every
// entry in the lane's stored order.
template <int M, int n>
static void check_butterflies(long* cases) {
  int v[M][n], st[M][n];
  for (int l = 0; l < M; ++l)
    for (int p = 0; p < n; ++p) v[l][p] = 1 + 7 * l + 131 * p + 3 * l * p;
  for (int l = 0; l < M; ++l)
    for (int s = 0; s < n; ++s) st[l][s] = v[l][s ^ ks_perm<M, n>(l)];
  int cur[M][n], len = n;
  for (int l = 0; l < M; ++l)
    for (int s = 0; s < n; ++s) cur[l][s] = st[l][s];
  for (int mask = M / 2; mask >= 1; mask /= 2) {  // reduce rounds, high lane bit first
    int nxt[M][n];
    for (int l = 0; l < M; ++l)
      for (int e = 0; e < len / 2; ++e) nxt[l][e] = cur[l][e] + cur[l ^ mask][len / 2 + e];
    len /= 2;
    for (int l = 0; l < M; ++l)
      for (int e = 0; e < len; ++e) cur[l][e] = nxt[l][e];
  }
  for (int l = 0; l < M; ++l)
    for (int e = 0; e < n / M; ++e) {
      int want = 0;
      for (int q = 0; q < M; ++q) want += v[q][(n / M) * l + e];
      ++*cases;
      if (cur[l][e] != want) { if (bad < 20) std::printf("FAIL reduce M=%d n=%d lane %d entry %d\n", M, n, l, e); ++bad; }
    }
  for (int mask = 1; mask < M; mask *= 2) {  // gather rounds, low lane bit first
    int nxt[M][n];
    for (int l = 0; l < M; ++l)
      for (int e = 0; e < len; ++e) { nxt[l][e] = cur[l][e]; nxt[l][len + e] = cur[l ^ mask][e]; }
    len *= 2;
    for (int l = 0; l < M; ++l)
      for (int e = 0; e < len; ++e) cur[l][e] = nxt[l][e];
  }
  for (int l = 0; l < M; ++l)
    for (int s = 0; s < n; ++s) {
      int want = 0;
      for (int q = 0; q < M; ++q) want += v[q][s ^ ks_perm<M, n>(l)];
      ++*cases;
      if (cur[l][s] != want) { if (bad < 20) std::printf("FAIL gather M=%d n=%d lane %d entry %d\n", M, n, l, s); ++bad; }
    }
}

int main() {
  long cases = 0;
  check_butterflies<2, 4>(&cases);
  check_butterflies<2, 8>(&cases);
  check_butterflies<4, 8>(&cases);
  check_butterflies<KS_NR, KS_TC>(&cases);
  check_butterflies<KS_NC, KS_TR>(&cases);
  const int nus[2] = {4, PDG_MODEL_NU_ALT};
  for (int a = 0; a < 2; ++a) {
    const int nu = nus[a];
    if (a == 1 && nu == 4) break;
    for (int N = 2; N <= NMAX; ++N) {
      for (int T = 64; T <= 576; T += 32) {
        const Lay L = make_lay(N, nu, T);
        if (L.ipw < 1) continue;  // the library rejects this CTA size
        ++cases;
        // image regions, in order, each as large as the kernels index it
        CHECK(NX - 1 <= 16, N, nu, T);  // x0 slots
        CHECK(L.x0 + 16 <= L.Xb && L.Xb + N * NX <= L.Ub && L.Ub + N * nu <= L.Am, N, nu, T);
        CHECK(L.Am + (N - 1) * STM_SAS <= L.Bm && L.Bm + (N - 1) * b_stride(nu) <= L.Bp, N, nu, T);
        CHECK(b_stride(nu) >= NX * nu && b_stride(nu) % 2 == 1, N, nu, T);
        CHECK(STM_SAS > make_stm_order().nnz && STM_SAS % 2 == 1 && make_stm_order().nnz <= NX * NX, N, nu, T);
        CHECK(L.Bp + (N - 1) * b_stride(nu) <= L.w && L.w + (N - 1) * NX <= L.eps, N, nu, T);
        CHECK(L.xh + N * NX <= L.uh && L.uh + N * nu <= L.mup && L.th + (N - 1) <= L.img, N, nu, T);
        // the phase-local union: PIPG form 1 and the discretization's stage buffers
        CHECK(L.img <= L.xt && L.td + N <= L.red, N, nu, T);
        CHECK(L.stage >= L.img && L.stage + L.ipw * L.sa <= L.red, N, nu, T);
        CHECK(L.sa == 2 * (SA_A + NX * nu) + 3 * NX, N, nu, T);
        // block reductions: K = 6 values per warp
        CHECK(6 * ((T + 31) / 32) <= L.total - L.red, N, nu, T);
        // PIPG form 2 (register blocks) where its thread rule is met
        if (T >= pipg_reg_threads(N, nu)) {
          const RegLay Q = make_reg_lay(L);
          CHECK(Q.vp >= L.img && Q.end <= L.red, N, nu, T);
          CHECK(Q.vp % 4 == 0 && Q.dx % 4 == 0 && Q.du % 4 == 0 && NXS % 4 == 0 && NXS >= NX, N, nu, T);
          CHECK(Q.dx - Q.vp == (N - 1) * NXS && Q.du - Q.dx == N * NXS && Q.td - Q.du >= N * nu, N, nu, T);
          CHECK(Q.end - Q.td >= N, N, nu, T);
        }
        // PIPG form 3 (register tiles over lane groups) where its thread rule is met
        if (T >= pipg_ks_threads(N) && T <= 512) {
          const KsLay Q = make_ks_lay(L);
          const int nup = KS_NC * ((nu + KS_NC - 1) / KS_NC);
          CHECK(KS_NXB >= NX && KS_NXB == KS_NR * KS_TR && KS_NXB == KS_NC * KS_TC, N, nu, T);
          CHECK(KS_GS * N <= T && nup >= nu && KS_TR % 2 == 0, N, nu, T);
          CHECK(Q.vp >= L.img && Q.end <= L.red, N, nu, T);
          CHECK(Q.vp % 4 == 0 && Q.dx % 4 == 0 && Q.du % 4 == 0 && Q.bq % 4 == 0 && Q.th % 4 == 0, N, nu, T);
          CHECK(Q.dx - Q.vp == N * KS_NXB && Q.du - Q.dx == N * KS_NXB, N, nu, T);
          CHECK(Q.bq - Q.du >= N * nup && Q.th - Q.bq >= N * nup && Q.end - Q.th >= N, N, nu, T);
        }
        // the adjoint's scratch, appended after the solve layout
        if (T == 256) {
          const AdjLay A = make_adj(L, nu, T);
          const int nm = (N - 1) * NX;
          CHECK(A.ss == L.dx - L.xt && A.Sb == L.total, N, nu, T);
          CHECK(A.Sb + A.ss <= A.rb && A.rb + nm <= A.hb && A.hb + N <= A.Gb, N, nu, T);
          CHECK(A.Gb + N * NX <= A.Gub && A.Gub + N * nu <= A.mup_m && A.mup_m + nm <= A.mum_m, N, nu, T);
          CHECK(A.mum_m + nm <= A.th_m && A.th_m + N <= A.u_m && A.u_m + N <= A.Xo, N, nu, T);
          CHECK(A.Xo + N * NX <= A.Uo && A.Uo + N * nu <= A.xob && A.xob + N * NX <= A.uob, N, nu, T);
          CHECK(A.uob + N * nu <= A.cA && A.cA + NX * NX <= A.cBm && A.cBm + NX * nu <= A.cBp, N, nu, T);
          CHECK(A.cBp + NX * nu <= A.cw && A.cw + NX <= A.gacc && A.gacc + (NX - 1) <= A.td, N, nu, T);
          CHECK(A.td + 4 * 32 * NX + SA_A + NX * nu <= A.tang, N, nu, T);
          // a record of one PIPG iteration for the reverse pass
          CHECK(A.sg == 3 * nm + N * NX + N * nu + (N - 1) + N, N, nu, T);
          const int groups = T / (NX + 2 * nu + 1);
          CHECK(groups >= 1 && A.tang + groups * 2 * (SA_A + NX * nu + 3 * NX) <= A.total, N, nu, T);
        }
      }
    }
  }
  if (bad) std::printf("FAILED %d of %ld cases\n", bad, cases);
  else std::printf("OK %ld\n", cases);
  return bad ? 1 : 0;
}
