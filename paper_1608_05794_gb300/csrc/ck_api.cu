// C ABI of the batched chemical-kinetics library (declared in include/ck.h).
// Host side: mechanism validation and packing (the paper's "binary
// database" of Sec. 5), host/device pointer handling, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ck.h"
#include "ck_internal.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? CK_ENOMEM : CK_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Device or host pointer?  Unregistered and pinned host memory are host.
bool is_host_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
}

int check_device(const ck_mech* m) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != m->hm.device)
    return fail(CK_EINVAL, "mechanism was loaded on device " + std::to_string(m->hm.device) +
                               " but the current device is " + std::to_string(dev));
  return CK_OK;
}

// Stage host arrays through device memory for one call.
struct Staged {
  struct Item {
    void* host;
    void* dev;
    size_t bytes;
    bool out;
  };
  std::vector<Item> items;
  cudaStream_t st;
  cudaError_t err = cudaSuccess;
  explicit Staged(cudaStream_t s) : st(s) {}
  template <class T>
  T* map(T* host, size_t count, bool in, bool out) {
    if (!host || count == 0) return host;
    void* d = nullptr;
    size_t bytes = count * sizeof(T);
    cudaError_t e = cudaMallocAsync(&d, bytes, st);
    if (e != cudaSuccess) {
      err = e;
      return nullptr;
    }
    if (in) {
      e = cudaMemcpyAsync(d, (const void*)host, bytes, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) err = e;
    }
    items.push_back({(void*)host, d, bytes, out});
    return static_cast<T*>(d);
  }
  cudaError_t finish() {
    cudaError_t e = err;
    for (auto& it : items)
      if (it.out && e == cudaSuccess) e = cudaMemcpyAsync(it.host, it.dev, it.bytes, cudaMemcpyDeviceToHost, st);
    for (auto& it : items) cudaFreeAsync(it.dev, st);
    cudaError_t s = cudaStreamSynchronize(st);
    return e != cudaSuccess ? e : s;
  }
};

bool finite(double x) { return std::isfinite(x); }

int validate(const ck_mech_desc* d) {
  if (!d) return fail(CK_EINVAL, "desc is NULL");
  const int S = d->n_species, R = d->n_reactions;
  if (S < 1 || S > CK_MAX_SPECIES) return fail(CK_ERANGE, "n_species must be in [1, 128]");
  if (R < 0 || R > CK_MAX_REACTIONS) return fail(CK_ERANGE, "n_reactions must be in [0, 32767]");
  if (!d->mw || !d->nasa || !d->t_mid) return fail(CK_EINVAL, "mw, nasa and t_mid are required");
  if (d->reactor != 0 && d->reactor != 1)
    return fail(CK_EINVAL, "reactor must be 0 (constant pressure) or 1 (constant volume)");
  if (R > 0 && (!d->reac || !d->prod || !d->arrh || !d->rtype || !d->reversible || !d->eff_ptr))
    return fail(CK_EINVAL, "reaction arrays are required when n_reactions > 0");
  for (int k = 0; k < S; ++k) {
    if (!(d->mw[k] > 0.0) || !finite(d->mw[k])) return fail(CK_EINVAL, "mw must be positive");
    if (!(d->t_mid[k] > 0.0) || !finite(d->t_mid[k])) return fail(CK_EINVAL, "t_mid must be positive");
    for (int c = 0; c < 14; ++c)
      if (!finite(d->nasa[k * 14 + c])) return fail(CK_EINVAL, "NASA-7 coefficients must be finite");
  }
  int n_eff = 0;
  for (int i = 0; i < R; ++i) {
    int nr = 0, np = 0;
    for (int s = 0; s < 3; ++s) {
      const int a = d->reac[i * 3 + s], b = d->prod[i * 3 + s];
      if (a < -1 || a >= S || b < -1 || b >= S)
        return fail(CK_EINVAL, "reaction " + std::to_string(i) + ": species index out of range");
      if (a >= 0) {
        if (nr != s) return fail(CK_EINVAL, "reaction " + std::to_string(i) + ": -1 padding must come last");
        ++nr;
      }
      if (b >= 0) {
        if (np != s) return fail(CK_EINVAL, "reaction " + std::to_string(i) + ": -1 padding must come last");
        ++np;
      }
    }
    if (nr == 0 || np == 0) return fail(CK_EINVAL, "reaction " + std::to_string(i) + ": empty side");
    const double* a = d->arrh + i * 3;
    if (!(a[0] > 0.0) || !finite(a[0]) || !finite(a[1]) || !finite(a[2]))
      return fail(CK_EINVAL, "reaction " + std::to_string(i) + ": Arrhenius A must be positive and finite");
    const int t = d->rtype[i];
    if (t < 0 || t > 2) return fail(CK_EINVAL, "reaction " + std::to_string(i) + ": rtype must be 0, 1 or 2");
    if (d->reversible[i] < 0 || d->reversible[i] > 2)
      return fail(CK_EINVAL, "reaction " + std::to_string(i) + ": reversible must be 0, 1 or 2");
    if (d->reversible[i] == 2) {
      if (!d->arrh_rev) return fail(CK_EINVAL, "arrh_rev is required for explicit reverse rates");
      const double* ar = d->arrh_rev + i * 3;
      if (!(ar[0] > 0.0) || !finite(ar[0]) || !finite(ar[1]) || !finite(ar[2]))
        return fail(CK_EINVAL, "reaction " + std::to_string(i) + ": reverse A must be positive and finite");
    }
    if (t == 2) {
      if (!d->arrh0) return fail(CK_EINVAL, "arrh0 is required for fall-off reactions");
      const double* a0 = d->arrh0 + i * 3;
      if (!(a0[0] > 0.0) || !finite(a0[0]) || !finite(a0[1]) || !finite(a0[2]))
        return fail(CK_EINVAL, "reaction " + std::to_string(i) + ": low-pressure A must be positive");
    }
    if (d->eff_ptr[i + 1] < d->eff_ptr[i]) return fail(CK_EINVAL, "eff_ptr must be non-decreasing");
    for (int e = d->eff_ptr[i]; e < d->eff_ptr[i + 1]; ++e) {
      if (!d->eff_sp || !d->eff_val) return fail(CK_EINVAL, "eff_sp/eff_val missing");
      if (d->eff_sp[e] < 0 || d->eff_sp[e] >= S) return fail(CK_EINVAL, "efficiency species out of range");
      if (!finite(d->eff_val[e]) || d->eff_val[e] < 0.0) return fail(CK_EINVAL, "efficiencies must be >= 0");
      if (t != 0 && d->eff_val[e] != 1.0) ++n_eff;
    }
    if (d->elem_count && d->n_elements > 0) {
      for (int el = 0; el < d->n_elements; ++el) {
        long bal = 0;
        for (int s = 0; s < 3; ++s) {
          if (d->reac[i * 3 + s] >= 0) bal -= d->elem_count[d->reac[i * 3 + s] * d->n_elements + el];
          if (d->prod[i * 3 + s] >= 0) bal += d->elem_count[d->prod[i * 3 + s] * d->n_elements + el];
        }
        if (bal != 0) return fail(CK_EINVAL, "reaction " + std::to_string(i) + " is not atom-balanced");
      }
    }
  }
  if (n_eff > 32767) return fail(CK_ERANGE, "too many third-body efficiencies");
  if (d->elem_count && d->elem_mass && d->n_elements > 0) {
    for (int k = 0; k < S; ++k) {
      long double w = 0.0L;
      for (int el = 0; el < d->n_elements; ++el)
        w += (long double)d->elem_count[k * d->n_elements + el] * d->elem_mass[el];
      if (std::fabs((double)(w - d->mw[k])) > 1e-12 * d->mw[k])
        return fail(CK_EINVAL, "mw of species " + std::to_string(k) + " differs from its composition");
    }
  }
  return CK_OK;
}

}  // namespace

int ck::set_error(int code, const char* msg) { return fail(code, msg); }

extern "C" {

void ck_default_opts(ck_solver_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->rtol = 1e-9;
  o->atol = 1e-12;
  o->max_steps = 100000;
}

int ck_load_mechanism(const ck_mech_desc* d, ck_mech** out) {
  using namespace ck;
  if (!out) return fail(CK_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(d);
  if (rc) return rc;
  const int S = d->n_species, R = d->n_reactions;
  const long double ln2 = 0.693147180559945309417232121458176568L;
  const long double Rg = 8.314462618L;
  // reactions, sorted by class so that neighbouring lanes of the team
  // kernels branch alike (the order of a sum over reactions changes only the
  // rounding of wdot)
  std::vector<int> order(R);
  for (int i = 0; i < R; ++i) order[i] = i;
  auto nside = [&](const int32_t* a, int i) {
    int c = 0;
    for (int s = 0; s < 3; ++s) c += a[i * 3 + s] >= 0;
    return c;
  };
  auto key = [&](int i) {
    return ((d->rtype[i] * 3 + d->reversible[i]) * 4 + nside(d->reac, i)) * 4 + nside(d->prod, i);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key(a) < key(b); });
  std::vector<RxnRec> rx(R);
  std::vector<int16_t> eff_sp;
  std::vector<double> eff_m1, revp;
  for (int ii = 0; ii < R; ++ii) {
    const int i = order[ii];
    RxnRec& r = rx[ii];
    std::memset(&r, 0, sizeof(r));
    const double* a = d->arrh + i * 3;
    r.lA2 = (double)(std::log2((long double)a[0]));
    r.beta = a[1];
    r.EoR2 = (double)((long double)a[2] / (Rg * ln2));
    r.type = (int8_t)d->rtype[i];
    r.rev = (int8_t)d->reversible[i];
    if (r.rev == 2) {
      const double* ar = d->arrh_rev + i * 3;
      r.rev_ix = (int16_t)(revp.size() / 3);
      revp.push_back((double)std::log2((long double)ar[0]));
      revp.push_back(ar[1]);
      revp.push_back((double)((long double)ar[2] / (Rg * ln2)));
    }
    if (r.type == 2) {
      const double* a0 = d->arrh0 + i * 3;
      r.lA02 = (double)(std::log2((long double)a0[0]));
      r.beta0 = a0[1];
      r.E0oR2 = (double)((long double)a0[2] / (Rg * ln2));
    }
    int nr = 0, np = 0;
    for (int s = 0; s < 3; ++s) {
      r.sp[s] = (int16_t)d->reac[i * 3 + s];
      r.sp[3 + s] = (int16_t)d->prod[i * 3 + s];
      nr += d->reac[i * 3 + s] >= 0;
      np += d->prod[i * 3 + s] >= 0;
    }
    r.nreac = (int8_t)nr;
    r.nprod = (int8_t)np;
    r.dnu = (int8_t)(np - nr);
    r.dnu_d = (double)(np - nr);
    r.nreac_d = (double)nr;
    r.nprod_d = (double)np;
    r.eff_beg = (int16_t)eff_sp.size();
    if (r.type != 0) {
      for (int e = d->eff_ptr[i]; e < d->eff_ptr[i + 1]; ++e) {
        if (d->eff_val[e] == 1.0) continue;
        eff_sp.push_back((int16_t)d->eff_sp[e]);
        eff_m1.push_back(d->eff_val[e] - 1.0);
      }
    }
    r.eff_cnt = (int16_t)(eff_sp.size() - r.eff_beg);
  }
  // thermo, pre-scaled (see ck_common.cuh for the layout)
  std::vector<double> th((size_t)S * TH_PER_SPECIES);
  for (int k = 0; k < S; ++k) {
    for (int rg = 0; rg < 2; ++rg) {
      const double* a = d->nasa + k * 14 + rg * 7;
      double* o = &th[(size_t)k * TH_PER_SPECIES + rg * TH_STRIDE];
      const long double a1 = a[0], a2 = a[1], a3 = a[2], a4 = a[3], a5 = a[4], a6 = a[5], a7 = a[6];
      o[0] = a[0]; o[1] = a[1]; o[2] = a[2]; o[3] = a[3]; o[4] = a[4];
      o[5] = a[0];
      o[6] = (double)(a2 / 2); o[7] = (double)(a3 / 3); o[8] = (double)(a4 / 4); o[9] = (double)(a5 / 5);
      o[10] = a[5];
      o[11] = (double)(a1 / ln2);
      o[12] = (double)((a7 - a1) / ln2);
      o[13] = (double)(a2 / (2 * ln2));
      o[14] = (double)(a3 / (6 * ln2));
      o[15] = (double)(a4 / (12 * ln2));
      o[16] = (double)(a5 / (20 * ln2));
      o[17] = (double)(-a6 / ln2);
    }
  }
  std::vector<double> W(d->mw, d->mw + S), invW(S), tmid(d->t_mid, d->t_mid + S);
  for (int k = 0; k < S; ++k) invW[k] = (double)(1.0L / (long double)d->mw[k]);
  std::vector<double> tab(256);
  for (int j = 0; j < 256; ++j) tab[j] = (double)std::exp2((long double)j / 256.0L);
  // species -> (reaction, net nu), in the sorted reaction order
  std::vector<int32_t> csr_ptr(S + 1, 0), csr_rx;
  std::vector<double> csr_nu;
  for (int k = 0; k < S; ++k) {
    csr_ptr[k] = (int32_t)csr_rx.size();
    for (int i = 0; i < R; ++i) {
      int nu = 0;
      for (int s = 0; s < 3; ++s) nu += (rx[i].sp[3 + s] == k) - (rx[i].sp[s] == k);
      if (nu != 0) {
        csr_rx.push_back(i);
        csr_nu.push_back((double)nu);
      }
    }
  }
  csr_ptr[S] = (int32_t)csr_rx.size();
  // team kernels walk the reactions in chunks of the CTA size
  const int chunk = (S + 1 <= 56) ? 64 : 256;
  const int n_chunks = (R + chunk - 1) / chunk;
  std::vector<int32_t> csr_cptr((size_t)S * (n_chunks + 1));
  for (int k = 0; k < S; ++k) {
    int e = csr_ptr[k];
    for (int c = 0; c <= n_chunks; ++c) {
      while (e < csr_ptr[k + 1] && csr_rx[e] < c * chunk) ++e;
      csr_cptr[(size_t)k * (n_chunks + 1) + c] = (c == n_chunks) ? csr_ptr[k + 1] : e;
    }
  }
  // Jacobian assembly, chunk by chunk, as one list of targets, each adding a
  // fixed-order sum of coef * src[pidx] (src: the chunk's per-reaction
  // arrays q, dq/dT, D and the partials P, contiguous in shared memory):
  // - species-block entries A[k][j] += nu_ki * P[i][slot] for every slot of
  //   reaction i holding species j (and nu_ki (eff_ij - 1) * P[i][6] for the
  //   third-body corrections), target index (1 + k) n + 1 + j;
  // - per species k the four sums over its reactions in the chunk, wdot_k
  //   (nu q), a_k (nu dq/dT), E_k (nu D) and u_k (nu P[i][6]), target index
  //   n^2 + a S + k for a = 0..3, terms in the CSR order.
  // Longest lists first, so that lanes running the same iteration do similar
  // amounts of work.
  std::vector<int32_t> jc_ptr(1, 0);
  std::vector<JcEntry> jc;
  std::vector<JcTerm> jt;
  int n_jterms = 0;
  const int NN = (S + 1) * (S + 1);
  for (int c = 0; c < n_chunks; ++c) {
    std::vector<std::vector<std::pair<double, int32_t>>> ent((size_t)S * S + 4 * (size_t)S);
    for (int k = 0; k < S; ++k) {
      for (int e = csr_cptr[(size_t)k * (n_chunks + 1) + c]; e < csr_cptr[(size_t)k * (n_chunks + 1) + c + 1];
           ++e) {
        const int i = csr_rx[e];
        const int li = i - c * chunk;
        const double nu = csr_nu[e];
        const RxnRec& r = rx[i];
        const int32_t pbase = 3 * chunk + li * JP;
        // coefficients carry W_k / W_j, the factor of the species block
        // dY_k/dY_j (so the assembly needs no per-entry rescaling)
        auto wr = [&](int j) { return (double)((long double)W[k] / (long double)W[j]); };
        for (int s2 = 0; s2 < r.nreac; ++s2)
          ent[(size_t)k * S + r.sp[s2]].push_back({nu * wr(r.sp[s2]), pbase + s2});
        if (r.rev)
          for (int s2 = 0; s2 < r.nprod; ++s2)
            ent[(size_t)k * S + r.sp[3 + s2]].push_back({nu * wr(r.sp[3 + s2]), pbase + 3 + s2});
        for (int q = r.eff_beg; q < r.eff_beg + r.eff_cnt; ++q)
          ent[(size_t)k * S + eff_sp[q]].push_back({nu * eff_m1[q] * wr(eff_sp[q]), pbase + 6});
        const size_t sb = (size_t)S * S;
        ent[sb + 0 * S + k].push_back({nu, li});
        ent[sb + 1 * S + k].push_back({nu, chunk + li});
        ent[sb + 2 * S + k].push_back({nu, 2 * chunk + li});
        ent[sb + 3 * S + k].push_back({nu, pbase + 6});
      }
    }
    std::vector<int> order_e;
    for (size_t e = 0; e < ent.size(); ++e)
      if (!ent[e].empty()) order_e.push_back((int)e);
    std::stable_sort(order_e.begin(), order_e.end(),
                     [&](int a, int b) { return ent[a].size() > ent[b].size(); });
    for (int e : order_e) {
      JcEntry h{};
      if (e < S * S) {
        const int k = e / S, j = e % S;
        h.idx = (1 + k) * (S + 1) + 1 + j;
        n_jterms += (int)ent[e].size();
      } else {
        h.idx = NN + (e - S * S);
      }
      h.beg = (int32_t)jt.size();
      for (auto& cc : ent[e]) {
        JcTerm t{};
        t.coef = cc.first;
        t.pidx = cc.second;
        jt.push_back(t);
      }
      h.end = (int32_t)jt.size();
      jc.push_back(h);
    }
    jc_ptr.push_back((int32_t)jc.size());
  }
  // species ordered by the length of their CSR rows (longest first), so
  // that the lanes of one warp gather similar counts in the one-pass RHS
  std::vector<int16_t> rsp(S);
  {
    std::vector<int> ks(S);
    for (int k = 0; k < S; ++k) ks[k] = k;
    std::stable_sort(ks.begin(), ks.end(), [&](int a, int b) {
      return csr_ptr[a + 1] - csr_ptr[a] > csr_ptr[b + 1] - csr_ptr[b];
    });
    for (int k = 0; k < S; ++k) rsp[k] = (int16_t)ks[k];
  }
  // one blob: staged block first, then the team-only tables
  StageLayout L{};
  size_t off = 0;
  auto place = [&](size_t bytes) {
    size_t o = off;
    off = align16(off + bytes);
    return (uint32_t)o;
  };
  L.rx = place(sizeof(RxnRec) * R);
  L.th = place(sizeof(double) * th.size());
  L.tmid = place(sizeof(double) * S);
  L.W = place(sizeof(double) * S);
  L.invW = place(sizeof(double) * S);
  L.eff_sp = place(sizeof(int16_t) * eff_sp.size());
  L.eff_m1 = place(sizeof(double) * eff_m1.size());
  L.revp = place(sizeof(double) * revp.size());
  L.tab = place(sizeof(double) * 256);
  L.bytes = (uint32_t)off;
  const size_t off_csr_ptr = place(sizeof(int32_t) * (S + 1));
  std::vector<CsrTerm> csr(csr_rx.size());
  for (size_t e = 0; e < csr.size(); ++e) {
    csr[e].nu = csr_nu[e];
    csr[e].rx = csr_rx[e];
    csr[e].pad = 0;
  }
  const size_t off_csr = place(sizeof(CsrTerm) * csr.size());
  const size_t off_csr_cptr = place(sizeof(int32_t) * csr_cptr.size());
  const size_t off_jc_ptr = place(sizeof(int32_t) * jc_ptr.size());
  const size_t off_jc = place(sizeof(JcEntry) * jc.size());
  const size_t off_jt = place(sizeof(JcTerm) * jt.size());
  const size_t off_rsp = place(sizeof(int16_t) * rsp.size());
  const size_t off_err = place(sizeof(int32_t) * 4);
  const size_t total = off;
  std::vector<unsigned char> host(total, 0);
  auto put = [&](size_t o, const void* src, size_t bytes) {
    if (bytes) std::memcpy(host.data() + o, src, bytes);
  };
  put(L.rx, rx.data(), sizeof(RxnRec) * R);
  put(L.th, th.data(), sizeof(double) * th.size());
  put(L.tmid, tmid.data(), sizeof(double) * S);
  put(L.W, W.data(), sizeof(double) * S);
  put(L.invW, invW.data(), sizeof(double) * S);
  put(L.eff_sp, eff_sp.data(), sizeof(int16_t) * eff_sp.size());
  put(L.eff_m1, eff_m1.data(), sizeof(double) * eff_m1.size());
  put(L.revp, revp.data(), sizeof(double) * revp.size());
  put(L.tab, tab.data(), sizeof(double) * 256);
  put(off_csr_ptr, csr_ptr.data(), sizeof(int32_t) * (S + 1));
  put(off_csr, csr.data(), sizeof(CsrTerm) * csr.size());
  put(off_csr_cptr, csr_cptr.data(), sizeof(int32_t) * csr_cptr.size());
  put(off_jc_ptr, jc_ptr.data(), sizeof(int32_t) * jc_ptr.size());
  put(off_jc, jc.data(), sizeof(JcEntry) * jc.size());
  put(off_jt, jt.data(), sizeof(JcTerm) * jt.size());
  put(off_rsp, rsp.data(), sizeof(int16_t) * rsp.size());

  ck_mech* m = new ck_mech;
  HostMech& hm = m->hm;
  cudaError_t e = cudaGetDevice(&hm.device);
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "cudaGetDevice");
  }
  e = cudaMalloc(&hm.blob, total);
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "cudaMalloc(mechanism tables)");
  }
  e = cudaMemcpy(hm.blob, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(hm.blob);
    delete m;
    return cuda_fail(e, "cudaMemcpy(mechanism tables)");
  }
  unsigned char* b = static_cast<unsigned char*>(hm.blob);
  hm.blob_bytes = total;
  hm.L = L;
  hm.S = S;
  hm.R = R;
  hm.rx = rx;
  DevMech& dm = hm.d;
  dm.S = S;
  dm.R = R;
  dm.n = S + 1;
  dm.n_eff = (int)eff_sp.size();
  dm.csr_nnz = (int)csr_rx.size();
  dm.rxn = reinterpret_cast<const RxnRec*>(b + L.rx);
  dm.thermo = reinterpret_cast<const double*>(b + L.th);
  dm.revp = reinterpret_cast<const double*>(b + L.revp);
  dm.cv = d->reactor;
  dm.tmid = reinterpret_cast<const double*>(b + L.tmid);
  dm.W = reinterpret_cast<const double*>(b + L.W);
  dm.invW = reinterpret_cast<const double*>(b + L.invW);
  dm.eff_sp = reinterpret_cast<const int16_t*>(b + L.eff_sp);
  dm.eff_m1 = reinterpret_cast<const double*>(b + L.eff_m1);
  dm.tab = reinterpret_cast<const double*>(b + L.tab);
  dm.csr_ptr = reinterpret_cast<const int32_t*>(b + off_csr_ptr);
  dm.csr = reinterpret_cast<const CsrTerm*>(b + off_csr);
  dm.chunk = chunk;
  dm.n_chunks = n_chunks;
  dm.csr_cptr = reinterpret_cast<const int32_t*>(b + off_csr_cptr);
  dm.jc_ptr = reinterpret_cast<const int32_t*>(b + off_jc_ptr);
  dm.jc = reinterpret_cast<const JcEntry*>(b + off_jc);
  dm.jt = reinterpret_cast<const JcTerm*>(b + off_jt);
  dm.rsp = reinterpret_cast<const int16_t*>(b + off_rsp);
  hm.n_contrib = n_jterms;
  hm.csr_nnz = (int)csr_rx.size();
  hm.dev_err = reinterpret_cast<int32_t*>(b + off_err);
  // resolve the allocation-free entry point's static scratch on this device
  // now, so that the driver's loading of the library's device code happens
  // in this call (which allocates anyway) and not in that entry point
  int32_t* scratch = nullptr;
  cudaError_t se = ck::noalloc_scratch(&scratch);
  if (se != cudaSuccess) {
    ck_free_mechanism(m);
    return cuda_fail(se, "cudaGetSymbolAddress(allocation-free scratch)");
  }
  *out = m;
  return CK_OK;
}

int ck_free_mechanism(ck_mech* m) {
  if (!m) return CK_OK;
  cudaError_t e = cudaSuccess;
  if (m->hm.blob) e = cudaFree(m->hm.blob);
  delete m;
  if (e != cudaSuccess) return cuda_fail(e, "cudaFree(mechanism tables)");
  return CK_OK;
}

int ck_mech_info(const ck_mech* m, int32_t* S, int32_t* R) {
  if (!m) return fail(CK_EINVAL, "mech is NULL");
  if (S) *S = m->hm.S;
  if (R) *R = m->hm.R;
  return CK_OK;
}

int ck_rhs(const ck_mech* m, int64_t n, const double* p, const double* y, double* dydt, void* stream) {
  if (!m) return fail(CK_EINVAL, "mech is NULL");
  if (n < 0) return fail(CK_EINVAL, "n < 0");
  if (n == 0) return CK_OK;
  if (!p || !y || !dydt) return fail(CK_EINVAL, "p, y and dydt are required");
  if (int rc = check_device(m)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nn = (size_t)m->hm.d.n;
  const bool host = is_host_ptr(p) || is_host_ptr(y) || is_host_ptr(dydt);
  if (!host) {
    cudaError_t e = ck::launch_rhs(m->hm, n, p, y, dydt, st);
    return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_rhs launch");
  }
  Staged sg(st);
  const double* dp = sg.map(const_cast<double*>(p), n, true, false);
  const double* dy = sg.map(const_cast<double*>(y), n * nn, true, false);
  double* df = sg.map(dydt, n * nn, false, true);
  if (sg.err == cudaSuccess) {
    cudaError_t e = ck::launch_rhs(m->hm, n, dp, dy, df, st);
    if (e != cudaSuccess) sg.err = e;
  }
  cudaError_t e = sg.finish();
  return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_rhs");
}

int ck_jacobian(const ck_mech* m, int64_t n, const double* p, const double* y, double* jac, void* stream) {
  if (!m) return fail(CK_EINVAL, "mech is NULL");
  if (n < 0) return fail(CK_EINVAL, "n < 0");
  if (n == 0) return CK_OK;
  if (!p || !y || !jac) return fail(CK_EINVAL, "p, y and jac are required");
  if (int rc = check_device(m)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nn = (size_t)m->hm.d.n;
  ck::LaunchCfg cfg;
  const bool host = is_host_ptr(p) || is_host_ptr(y) || is_host_ptr(jac);
  if (!host) {
    cudaError_t e = ck::launch_jacobian(m->hm, n, p, y, jac, st, cfg);
    return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_jacobian launch");
  }
  Staged sg(st);
  const double* dp = sg.map(const_cast<double*>(p), n, true, false);
  const double* dy = sg.map(const_cast<double*>(y), n * nn, true, false);
  double* dj = sg.map(jac, n * nn * nn, false, true);
  if (sg.err == cudaSuccess) {
    cudaError_t e = ck::launch_jacobian(m->hm, n, dp, dy, dj, st, cfg);
    if (e != cudaSuccess) sg.err = e;
  }
  cudaError_t e = sg.finish();
  return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_jacobian");
}

int ck_jacobian_fd(const ck_mech* m, int64_t n, const double* p, const double* y, const double* h, double rtol,
                   double atol, double* jac, void* stream) {
  if (!m) return fail(CK_EINVAL, "mech is NULL");
  if (n < 0) return fail(CK_EINVAL, "n < 0");
  if (n == 0) return CK_OK;
  if (!p || !y || !h || !jac) return fail(CK_EINVAL, "p, y, h and jac are required");
  if (!(rtol > 0.0) || !(atol > 0.0)) return fail(CK_EINVAL, "need rtol > 0 and atol > 0");
  if (int rc = check_device(m)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nn = (size_t)m->hm.d.n;
  ck::LaunchCfg cfg;
  const bool host = is_host_ptr(p) || is_host_ptr(y) || is_host_ptr(h) || is_host_ptr(jac);
  if (!host) {
    cudaError_t e = ck::launch_jacobian_fd(m->hm, n, p, y, h, rtol, atol, jac, st, cfg);
    return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_jacobian_fd launch");
  }
  Staged sg(st);
  const double* dp = sg.map(const_cast<double*>(p), n, true, false);
  const double* dy = sg.map(const_cast<double*>(y), n * nn, true, false);
  const double* dh = sg.map(const_cast<double*>(h), n, true, false);
  double* dj = sg.map(jac, n * nn * nn, false, true);
  if (sg.err == cudaSuccess) {
    cudaError_t e = ck::launch_jacobian_fd(m->hm, n, dp, dy, dh, rtol, atol, dj, st, cfg);
    if (e != cudaSuccess) sg.err = e;
  }
  cudaError_t e = sg.finish();
  return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_jacobian_fd");
}

int ck_lu_factor(int64_t batch, int32_t dim, double* a, int32_t* piv, int32_t* info, void* stream) {
  if (batch < 0 || dim < 1 || dim > 128) return fail(CK_ERANGE, "need batch >= 0 and 1 <= dim <= 128");
  if (batch == 0) return CK_OK;
  if (!a || !piv || !info) return fail(CK_EINVAL, "a, piv and info are required");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool host = is_host_ptr(a) || is_host_ptr(piv) || is_host_ptr(info);
  if (!host) {
    cudaError_t e = ck::launch_lu_factor(batch, dim, a, piv, info, st);
    return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_lu_factor launch");
  }
  Staged sg(st);
  double* da = sg.map(a, (size_t)batch * dim * dim, true, true);
  int32_t* dp = sg.map(piv, (size_t)batch * dim, false, true);
  int32_t* di = sg.map(info, (size_t)batch, false, true);
  if (sg.err == cudaSuccess) {
    cudaError_t e = ck::launch_lu_factor(batch, dim, da, dp, di, st);
    if (e != cudaSuccess) sg.err = e;
  }
  cudaError_t e = sg.finish();
  return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_lu_factor");
}

int ck_lu_solve(int64_t batch, int32_t dim, const double* lu, const int32_t* piv, double* b, void* stream) {
  if (batch < 0 || dim < 1 || dim > 128) return fail(CK_ERANGE, "need batch >= 0 and 1 <= dim <= 128");
  if (batch == 0) return CK_OK;
  if (!lu || !piv || !b) return fail(CK_EINVAL, "lu, piv and b are required");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool host = is_host_ptr(lu) || is_host_ptr(piv) || is_host_ptr(b);
  if (!host) {
    cudaError_t e = ck::launch_lu_solve(batch, dim, lu, piv, b, st);
    return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_lu_solve launch");
  }
  Staged sg(st);
  const double* dl = sg.map(const_cast<double*>(lu), (size_t)batch * dim * dim, true, false);
  const int32_t* dp = sg.map(const_cast<int32_t*>(piv), (size_t)batch * dim, true, false);
  double* db = sg.map(b, (size_t)batch * dim, true, true);
  if (sg.err == cudaSuccess) {
    cudaError_t e = ck::launch_lu_solve(batch, dim, dl, dp, db, st);
    if (e != cudaSuccess) sg.err = e;
  }
  cudaError_t e = sg.finish();
  return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_lu_solve");
}

}  // extern "C"

namespace {

// RKF45 mapping: explicit form, else one CTA per reactor unless the
// mechanism is small (per-lane scratch stays on chip) and the batch fills
// every SM with four 128-thread blocks of one reactor per thread.
bool rkf45_team(const ck::HostMech& hm, int form, int64_t n) {
  if (form == 1) return false;
  if (form == 2) return true;
  return hm.S > 32 || n < (int64_t)4 * 128 * ck::sm_count();
}

int integrate(int method, const ck_mech* m, int64_t n, const double* p, double* y, const double* dt,
              double* h_io, const ck_solver_opts* opts, int32_t* steps, int32_t* status, void* stream) {
  if (n < 0 || n > CK_MAX_REACTORS) return fail(CK_ERANGE, "n must be in [0, CK_MAX_REACTORS = 2^30]");
  if (!m) return fail(CK_EINVAL, "mech is NULL");
  if (n == 0) return CK_OK;
  if (!p || !y || !dt || !status) return fail(CK_EINVAL, "p, y, dt and status are required");
  ck_solver_opts o;
  if (opts) o = *opts;
  else ck_default_opts(&o);
  if (!(o.rtol > 0.0) || !(o.atol > 0.0) || o.max_steps < 1 || !(o.h0 >= 0.0) || !(o.fixed_h >= 0.0))
    return fail(CK_EINVAL, "opts: need rtol > 0, atol > 0, max_steps >= 1, h0 >= 0, fixed_h >= 0");
  if (o.precision < 0 || o.precision > 2 || (o.precision != 0 && method != 0))
    return fail(CK_EINVAL, "opts.precision: 0 (FP64) for both methods; 1 or 2 (FP32 LU + 1 or 2 FP64 "
                           "refinement steps) for ROS4");
  if (o.form < 0 || o.form > 2) return fail(CK_EINVAL, "opts.form must be 0, 1 or 2");
  if (!(o.team == 0 || o.team == 8 || o.team == 16)) return fail(CK_EINVAL, "opts.team must be 0, 8 or 16");
  if (o.jac < 0 || o.jac > 1 || (o.jac != 0 && method != 0))
    return fail(CK_EINVAL, "opts.jac: 0 (analytic) for both methods; 1 (forward differences) for ROS4");
  if (int rc = check_device(m)) return rc;
  ck::SolverParams sp{o.rtol, o.atol, o.h0, o.fixed_h, o.max_steps, o.jac};
  ck::LaunchCfg cfg;
  if (o.variant > 0) cfg.ctas_per_sm = o.variant;
  cfg.precision = o.precision;
  cfg.grid_side = o.team;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nn = (size_t)m->hm.d.n;
  const bool host = is_host_ptr(p) || is_host_ptr(y) || is_host_ptr(dt) || is_host_ptr(h_io) ||
                    is_host_ptr(steps) || is_host_ptr(status);
  Staged sg(st);
  const double* dp = p;
  double* dy = y;
  const double* ddt = dt;
  double* dh = h_io;
  int32_t* ds = steps;
  int32_t* dst = status;
  if (host) {
    dp = sg.map(const_cast<double*>(p), n, true, false);
    dy = sg.map(y, n * nn, true, true);
    ddt = sg.map(const_cast<double*>(dt), n, true, false);
    dh = sg.map(h_io, n, true, true);
    ds = sg.map(steps, 2 * n, false, true);
    dst = sg.map(status, n, false, true);
    if (sg.err != cudaSuccess) {
      sg.finish();
      return cuda_fail(sg.err, "staging host arrays");
    }
  }
  int32_t* queue = nullptr;
  cudaError_t e = cudaMallocAsync(&queue, sizeof(int32_t), st);
  if (e == cudaSuccess) {
    if (method == 0)
      e = ck::launch_ros4(m->hm, n, dp, dy, ddt, dh, sp, ds, dst, queue, st, cfg, nullptr, 0, true);
    else if (rkf45_team(m->hm, o.form, n))
      e = ck::launch_rkf45_team(m->hm, n, dp, dy, ddt, dh, sp, ds, dst, queue, st, cfg);
    else
      e = ck::launch_rkf45(m->hm, n, dp, dy, ddt, dh, sp, ds, dst, queue, st, cfg);
    cudaFreeAsync(queue, st);
  }
  if (host) {
    if (e != cudaSuccess) sg.err = e;
    e = sg.finish();
  }
  return e == cudaSuccess ? CK_OK : cuda_fail(e, method == 0 ? "ck_integrate_ros4" : "ck_integrate_rkf45");
}

// FP64 instruction counts of this library's formulation (see ck.h).
double rhs_count(const ck::HostMech& hm) {
  // species pass: mixture, NASA-7 polynomials and the two Gibbs factors
  // 2^(+-g_k) (8 each) per species
  double c = 20.0 + 40.0 * hm.S;
  for (const auto& r : hm.rx) {
    c += 2 + 8 + (r.nreac - 1) + 1 + (r.nreac + r.nprod);
    // 1/K_c as a product of species factors, then k_r and the reverse product
    if (r.rev == 1) c += 1 + (r.nreac + r.nprod) + 1 + (r.nprod - 1) + 1;
    if (r.rev == 2) c += 2 + 8 + (r.nprod - 1) + 1;
    if (r.type) c += r.eff_cnt + 1;
    if (r.type == 2) c += 2 + 1 + 8 + 1 + 1 + 1 + 1;
  }
  return c;
}
double rhs_exps(const ck::HostMech& hm) {
  double c = 2.0 * hm.S;  // 2^(+-g_k) per species
  for (const auto& r : hm.rx) c += 1 + (r.rev == 2 ? 1 : 0) + (r.type == 2 ? 1 : 0);
  return c;
}
double jac_count(const ck::HostMech& hm) {
  const double S = hm.S;
  // species pass extras (dcp), the species-block zeroing is not FP64,
  // column sums S^2, dense row terms S^2, temperature row / column 14 S, J00
  double c = 4.0 * S + S * S + S * S + 14.0 * S + 30.0;
  for (const auto& r : hm.rx) {
    double per = 3 + 3 + 4 + 1 + 6 + 1;  // dlnkf, c k, w, D, dq/dT
    if (r.rev == 1) per += (r.nreac + r.nprod) + 2;
    if (r.rev == 2) per += 2;
    if (r.type == 2) per += 7;
    per += (r.nreac == 2 ? 2 : (r.nreac == 3 ? 6 : 0));
    if (r.rev) per += (r.nprod == 2 ? 2 : (r.nprod == 3 ? 6 : 1));
    c += per;
  }
  c += hm.n_contrib;          // one FMA per contribution
  c += 3.0 * hm.csr_nnz;      // aT, E, u (wdot is counted in the RHS)
  return c;
}
// The same units in the flop model of the roofline (an FMA counts 2 flops,
// any other FP64 add, multiply, divide or comparison 1; exponentials and
// logarithms are counted apart, as transcendentals): the algorithm's
// arithmetic, without the reduction trees, predicated lanes and index work of
// its GPU mapping.
struct Ops {
  double fma = 0, other = 0, transc = 0;
  double flops() const { return 2.0 * fma + other; }
};

Ops rhs_ops(const ck::HostMech& hm) {
  Ops o;
  const double S = hm.S;
  const bool cv = hm.d.cv != 0;
  o.other += cv ? 7 : 9;  // 1/T, log2 T, T^2..T^4, 1/sum(Y/W), rho
  o.transc += 1;          // ln T
  o.fma += 16 * S;        // sum Y/W, Gibbs (6), cp (4) and H (5) polynomials
  o.other += 3 * S;       // [X_k] (2), C (1)
  o.transc += 2 * S;      // 2^(+-g_k)
  o.fma += 2 * S;         // cp mixture, sum H wdot
  o.other += 3 * S + (cv ? 2 * S : 0) + 4;  // Y/W, W/rho, dY/dt; U = H - RT; 1/rho, dT/dt
  for (const auto& r : hm.rx) {
    o.fma += 2;           // log2 k_f
    o.transc += 1;        // k_f
    o.other += r.nreac - 1;  // forward product
    if (r.rev == 1) {
      o.other += (r.nreac + r.nprod) - (r.dnu == 0 ? 1 : 0) + (std::abs((int)r.dnu) == 2 ? 1 : 0) + 1 + (r.nprod - 1);
      o.other += 1;
      o.fma += 1;         // q = k_f prod' - k_r prod''
    } else if (r.rev == 2) {
      o.fma += 2;
      o.transc += 1;
      o.other += (r.nprod - 1) + 1;
      o.fma += 1;
    } else {
      o.other += 1;
    }
    if (r.type) {
      o.fma += r.eff_cnt;  // [M]
      o.other += 1;        // q = c net
    }
    if (r.type == 2) {
      o.fma += 2;
      o.transc += 1;
      o.other += 5;        // k0/k_inf exponent, P_r, 1 + P_r, 1/(1 + P_r), c
    }
  }
  o.fma += hm.csr_nnz;    // wdot_k = sum nu q
  return o;
}

Ops jac_ops(const ck::HostMech& hm) {
  Ops o;
  const double S = hm.S;
  o.fma += 4 * S;         // d cp_mix / dT
  o.other += 4 * S;
  for (const auto& r : hm.rx) {
    o.fma += 1;           // d ln k_f / dT
    o.other += 2;
    if (r.rev == 1) o.other += r.nreac + r.nprod + 1;      // d ln K_c / dT
    if (r.rev == 2) {
      o.fma += 1;
      o.other += 3;
    }
    if (r.type == 2) {
      o.fma += 1;
      o.other += 8;       // d ln k0/dT, dc/dT, dc/d[M]
    }
    o.other += 2 + (r.type ? 1 : 0);  // c k_f, c k_r, dc/d[M] net
    o.other += (r.nreac == 2 ? 2 : (r.nreac == 3 ? 6 : 0));
    if (r.rev) o.other += (r.nprod == 2 ? 2 : (r.nprod == 3 ? 6 : 0));
    o.fma += r.type ? 2 : 1;  // D (Euler sum)
    o.other += 3;
    o.other += 4;             // dq/dT at fixed [X]
    if (r.type == 2) o.fma += 1;
    if (!hm.d.cv) o.fma += 1; // at fixed Y
  }
  o.fma += hm.n_contrib;        // species block contributions
  o.fma += 3.0 * hm.csr_nnz;    // d wdot/dT, E, u
  o.fma += 5 * S;               // column-sum and dense-row terms
  o.other += 4 * S;
  o.fma += S * S + S;           // temperature-row column sums
  o.fma += S * S;               // dense part of the species block
  o.fma += S;                   // temperature column
  o.other += 3 * S;
  o.fma += 2 * S;               // temperature row
  o.other += 6 * S;
  o.fma += 2;                   // J_00
  o.other += 15;
  return o;
}

Ops lu_ops(int n) {
  Ops o;
  for (int k = 0; k < n; ++k) {
    const double m = n - k - 1;
    o.other += 1 + m;       // reciprocal pivot, multipliers
    o.fma += m * m;         // rank-one update
  }
  return o;
}

Ops solve_ops(int n) {
  Ops o;
  o.fma = (double)n * (n - 1);  // forward and back substitution
  o.other = n;                  // diagonal
  return o;
}

double lu_count(int n) {
  double c = 0.0;
  for (int k = 0; k < n; ++k) c += 1 + (n - k - 1) + (double)(n - k - 1) * (n - k - 1);
  return c;
}

}  // namespace

extern "C" {

int ck_integrate_ros4(const ck_mech* m, int64_t n, const double* p, double* y, const double* dt,
                      double* h_inout, const ck_solver_opts* opts, int32_t* steps, int32_t* status,
                      void* stream) {
  return integrate(0, m, n, p, y, dt, h_inout, opts, steps, status, stream);
}

int ck_integrate_rkf45(const ck_mech* m, int64_t n, const double* p, double* y, const double* dt,
                       double* h_inout, const ck_solver_opts* opts, int32_t* steps, int32_t* status,
                       void* stream) {
  return integrate(1, m, n, p, y, dt, h_inout, opts, steps, status, stream);
}

int ck_integrate_ros4_noalloc(const ck_mech* m, int64_t n, const double* p, double* y,
                              const double* dt, double* h_inout, const ck_solver_opts* opts,
                              int32_t* steps, int32_t* status, void* stream) {
  if (n < 0) return fail(CK_EINVAL, "n < 0");
  if (n > CK_NOALLOC_MAX_REACTORS)
    return fail(CK_ERANGE, "ck_integrate_ros4_noalloc: n = " + std::to_string(n) +
                               " exceeds CK_NOALLOC_MAX_REACTORS (" +
                               std::to_string((long long)CK_NOALLOC_MAX_REACTORS) +
                               "); split the batch into several calls");
  if (!m) return fail(CK_EINVAL, "mech is NULL");
  if (n == 0) return CK_OK;
  if (!p || !y || !dt || !status) return fail(CK_EINVAL, "p, y, dt and status are required");
  if (is_host_ptr(p) || is_host_ptr(y) || is_host_ptr(dt) || is_host_ptr(h_inout) ||
      is_host_ptr(steps) || is_host_ptr(status))
    return fail(CK_EINVAL,
                "ck_integrate_ros4_noalloc takes device pointers only: host arrays would need "
                "device staging buffers, which this entry point does not allocate");
  ck_solver_opts o;
  if (opts) o = *opts;
  else ck_default_opts(&o);
  if (!(o.rtol > 0.0) || !(o.atol > 0.0) || o.max_steps < 1 || !(o.h0 >= 0.0) || !(o.fixed_h >= 0.0))
    return fail(CK_EINVAL, "opts: need rtol > 0, atol > 0, max_steps >= 1, h0 >= 0, fixed_h >= 0");
  if (o.precision != 0) return fail(CK_EINVAL, "opts.precision: only 0 (FP64) is available");
  if (o.jac < 0 || o.jac > 1) return fail(CK_EINVAL, "opts.jac must be 0 or 1");
  if (!(o.team == 0 || o.team == 8 || o.team == 16)) return fail(CK_EINVAL, "opts.team must be 0, 8 or 16");
  if (int rc = check_device(m)) return rc;
  ck::SolverParams sp{o.rtol, o.atol, o.h0, o.fixed_h, o.max_steps, o.jac};
  ck::LaunchCfg cfg;
  if (o.variant > 0) cfg.ctas_per_sm = o.variant;
  cfg.grid_side = o.team;
  cudaError_t e = ck::launch_ros4_noalloc(m->hm, n, p, y, dt, h_inout, sp, steps, status,
                                         static_cast<cudaStream_t>(stream), cfg);
  return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_integrate_ros4_noalloc");
}

int ck_count_work(const ck_mech* m, ck_work_counts* o) {
  if (!m || !o) return fail(CK_EINVAL, "mech and out are required");
  const ck::HostMech& hm = m->hm;
  const int n = hm.S + 1;
  o->rhs_fp64 = rhs_count(hm);
  o->rhs_exps = rhs_exps(hm);
  o->jac_fp64 = jac_count(hm);
  o->lu_fp64 = lu_count(n);
  o->solve_fp64 = (double)n * n;
  o->ros4_step_fp64 = o->jac_fp64 + 3.0 * o->rhs_fp64 + o->lu_fp64 + 4.0 * o->solve_fp64 +
                      (double)n * n + 30.0 * n;
  o->rkf45_step_fp64 = 6.0 * o->rhs_fp64 + 40.0 * n;
  // f(y), n difference columns (each an RHS, a subtract and a divide per
  // entry), the fnorm and increments, then stages 2 and 3 as above
  o->ros4_fd_step_fp64 = (n + 3.0) * o->rhs_fp64 + 2.0 * (double)n * n + 8.0 * n + o->lu_fp64 +
                         4.0 * o->solve_fp64 + (double)n * n + 30.0 * n;
  o->rhs_bytes = 8.0 * (2 * n + 1);
  o->integrate_bytes = 8.0 * (2 * n + 2) + 4.0;
  const Ops rh = rhs_ops(hm), jc = jac_ops(hm), lu = lu_ops(n), so = solve_ops(n);
  o->rhs_flops = rh.flops();
  o->rhs_transc = rh.transc;
  o->jac_flops = jc.flops();
  o->lu_flops = lu.flops();
  o->solve_flops = so.flops();
  // ROS4 attempt: stage vectors, update, error and norm (18 FMAs and 4 other
  // operations a component) and the diagonal of the iteration matrix
  const double ros_vec = 2.0 * 18 * n + 4.0 * n + 20;
  o->ros4_jeval_flops = jc.flops() + rh.flops();
  o->ros4_attempt_flops = 2.0 * rh.flops() + lu.flops() + 4.0 * so.flops() + ros_vec;
  o->ros4_step_flops = o->ros4_jeval_flops + o->ros4_attempt_flops;
  // RKF45 step: six stages, update, error and norm (25 FMAs and 9 other
  // operations a component)
  o->rkf45_step_flops = 6.0 * rh.flops() + 2.0 * 25 * n + 9.0 * n + 20;
  // forward-difference Jacobian: f(y), n columns (each an RHS, a difference
  // and a quotient a component), the increments and fnorm
  o->ros4_fd_jeval_flops = (n + 1.0) * rh.flops() + 2.0 * (double)n * n + 8.0 * n;
  return CK_OK;
}

int ck_device_errors(const ck_mech* m, int32_t* bits, int32_t reset) {
  if (!m || !bits) return fail(CK_EINVAL, "mech and bits are required");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(bits, m->hm.dev_err, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(m->hm.dev_err, 0, sizeof(int32_t));
  return e == cudaSuccess ? CK_OK : cuda_fail(e, "ck_device_errors");
}

const char* ck_status_str(int code) {
  switch (code) {
    case CK_OK: return "ok";
    case CK_EINVAL: return "invalid argument";
    case CK_ECUDA: return "CUDA error";
    case CK_ENOMEM: return "out of device memory";
    case CK_AGAIN: return "resource temporarily insufficient";
    case CK_TIMEOUT: return "bounded device wait gave up";
    case CK_ERANGE: return "size beyond a documented limit";
    default: return "unknown status";
  }
}

const char* ck_last_error(void) { return g_err.c_str(); }

const char* ck_version(void) { return "ck 0.1 (sm_103a, FP64)"; }

}  // extern "C"
