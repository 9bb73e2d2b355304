// BP error estimate of one edge (Methods, "Estimating the error of BP for
// general tensor networks", Eq. BPErrorEstimate): the norm network of the
// state in the symmetric gauge, cut along the edge, is contracted exactly down
// to the chi^2 x chi^2 edge environment E; BP takes E as rank one, and the
// error estimate is 1 - sqrt(s_1^2 / sum_i s_i^2) over E's singular values.
//
// Host FP64.  The symmetric gauge is the Vidal gauge with lambda^1/2 on every
// leg (tn_vidal_gauge, on the device); each site's double-layer tensor
// D_v[(l, l'), ..] = sum_p T[p, l, ..] conj(T[p, l', ..]) keeps only the
// support of each lambda_e; the cut edge's index is split into a u-side and a
// w-side label; the network is contracted pairwise, always taking the pair
// with the smallest result (a greedy order), and refused once an intermediate
// would exceed kMaxElems elements.  E^H E is diagonalised by cyclic Jacobi.
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <string>
#include <vector>

#include "tnbp.h"

namespace tnbp {
void set_error(const std::string& m);  // the thread's tn_last_error message
}

namespace {

using cplx = std::complex<double>;
constexpr int64_t kMaxElems = int64_t(1) << 26;

struct Tensor {
  std::vector<int> lab;      // one label per index
  std::vector<int64_t> dim;  // its dimension
  std::vector<cplx> a;       // row-major over the indices in order
  int64_t size() const {
    int64_t s = 1;
    for (int64_t d : dim) s *= d;
    return s;
  }
};

// t with its indices reordered to `order` (a permutation of positions).
Tensor permute(const Tensor& t, const std::vector<int>& order) {
  const int r = (int)order.size();
  Tensor o;
  o.lab.resize(r);
  o.dim.resize(r);
  for (int i = 0; i < r; ++i) { o.lab[i] = t.lab[order[i]]; o.dim[i] = t.dim[order[i]]; }
  std::vector<int64_t> st(r, 1);  // strides of t
  for (int i = r - 2; i >= 0; --i) st[i] = st[i + 1] * t.dim[i + 1];
  o.a.resize(t.a.size());
  std::vector<int64_t> idx(r, 0);
  for (int64_t n = 0; n < (int64_t)o.a.size(); ++n) {
    int64_t src = 0;
    for (int i = 0; i < r; ++i) src += idx[i] * st[order[i]];
    o.a[n] = t.a[src];
    for (int i = r - 1; i >= 0; --i) {
      if (++idx[i] < o.dim[i]) break;
      idx[i] = 0;
    }
  }
  return o;
}

// Contract the labels x and y share: result indices x-only then y-only.
Tensor contract(const Tensor& x, const Tensor& y) {
  std::vector<int> xs, xk, ys, yk;  // x: kept / shared positions, y: shared / kept
  for (int i = 0; i < (int)x.lab.size(); ++i) {
    const auto it = std::find(y.lab.begin(), y.lab.end(), x.lab[i]);
    (it == y.lab.end() ? xk : xs).push_back(i);
  }
  for (int s : xs) ys.push_back((int)(std::find(y.lab.begin(), y.lab.end(), x.lab[s]) - y.lab.begin()));
  for (int i = 0; i < (int)y.lab.size(); ++i)
    if (std::find(ys.begin(), ys.end(), i) == ys.end()) yk.push_back(i);
  std::vector<int> ox(xk), oy(ys);
  ox.insert(ox.end(), xs.begin(), xs.end());
  oy.insert(oy.end(), yk.begin(), yk.end());
  const Tensor px = permute(x, ox), py = permute(y, oy);
  int64_t m = 1, k = 1, n = 1;
  for (int i : xk) m *= x.dim[i];
  for (int i : xs) k *= x.dim[i];
  for (int i : yk) n *= y.dim[i];
  Tensor o;
  for (int i : xk) { o.lab.push_back(x.lab[i]); o.dim.push_back(x.dim[i]); }
  for (int i : yk) { o.lab.push_back(y.lab[i]); o.dim.push_back(y.dim[i]); }
  o.a.assign(m * n, cplx(0.0, 0.0));
  for (int64_t i = 0; i < m; ++i)
    for (int64_t q = 0; q < k; ++q) {
      const cplx xv = px.a[i * k + q];
      if (xv == cplx(0.0, 0.0)) continue;
      const cplx* yr = &py.a[q * n];
      cplx* orow = &o.a[i * n];
      for (int64_t j = 0; j < n; ++j) orow[j] += xv * yr[j];
    }
  return o;
}

int64_t result_size(const Tensor& x, const Tensor& y) {
  int64_t s = 1;
  for (size_t i = 0; i < x.lab.size(); ++i)
    if (std::find(y.lab.begin(), y.lab.end(), x.lab[i]) == y.lab.end()) s *= x.dim[i];
  for (size_t i = 0; i < y.lab.size(); ++i)
    if (std::find(x.lab.begin(), x.lab.end(), y.lab[i]) == x.lab.end()) s *= y.dim[i];
  return s;
}

bool shares(const Tensor& x, const Tensor& y) {
  for (int l : x.lab)
    if (std::find(y.lab.begin(), y.lab.end(), l) != y.lab.end()) return true;
  return false;
}

// Eigenvalues of the Hermitian n x n matrix h (row-major, destroyed), cyclic Jacobi.
std::vector<double> hermitian_eigenvalues(std::vector<cplx>& h, int n) {
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double a2 = std::norm(h[(size_t)i * n + j]);
        tot += a2;
        if (i != j) off += a2;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cplx c = h[(size_t)p * n + q];
        const double r = std::abs(c);
        if (r < 1e-300) continue;
        const double a = h[(size_t)p * n + p].real(), b = h[(size_t)q * n + q].real();
        const cplx ph = std::conj(c) / r;  // e^{-i phi}
        const double tau = (b - a) / (2.0 * r);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        // columns p, q: A J with J = [[cs, sn], [-sn ph, cs ph]]
        for (int i = 0; i < n; ++i) {
          const cplx aip = h[(size_t)i * n + p], aiq = ph * h[(size_t)i * n + q];
          h[(size_t)i * n + p] = cs * aip - sn * aiq;
          h[(size_t)i * n + q] = sn * aip + cs * aiq;
        }
        // rows p, q: J^H A
        for (int j = 0; j < n; ++j) {
          const cplx apj = h[(size_t)p * n + j], aqj = std::conj(ph) * h[(size_t)q * n + j];
          h[(size_t)p * n + j] = cs * apj - sn * aqj;
          h[(size_t)q * n + j] = sn * apj + cs * aqj;
        }
      }
  }
  std::vector<double> ev(n);
  for (int i = 0; i < n; ++i) ev[i] = h[(size_t)i * n + i].real();
  return ev;
}

}  // namespace

extern "C" tn_status tn_bp_error(tn_handle* h, int32_t e, double* error, double* sv_out,
                                 int32_t sv_capacity, int32_t* n_sv) {
  if (!h || !error) { tnbp::set_error("null argument"); return TN_EINVAL; }
  int32_t n = 0, m = 0, chi = 0;
  tn_status st = tn_graph_info(h, &n, &m, &chi, nullptr, 0);
  if (st) return st;
  if (e < 0 || e >= m) { tnbp::set_error("edge out of range"); return TN_EINVAL; }
  std::vector<int32_t> edges(2 * (size_t)m);
  st = tn_graph_info(h, &n, &m, &chi, edges.data(), m);
  if (st) return st;
  std::vector<double> lam((size_t)m * chi);
  st = tn_vidal_gauge(h, lam.data());
  if (st) return st;
  // support of each bond and the legs of each site in increasing edge id
  std::vector<int> rsup(m, 0);
  for (int f = 0; f < m; ++f)
    for (int k = 0; k < chi; ++k)
      if (lam[(size_t)f * chi + k] > 0.0) rsup[f] = k + 1;
  std::vector<std::vector<int>> legs(n);
  for (int f = 0; f < m; ++f) {
    legs[edges[2 * f]].push_back(f);
    legs[edges[2 * f + 1]].push_back(f);
  }
  // double-layer tensors of the symmetric gauge, bonds cut to the supports;
  // labels: edge f -> f, the cut edge's u side -> m, w side -> m + 1
  // the double-layer tensors together stay within 2 x kMaxElems elements
  {
    double total = 0.0;
    for (int v = 0; v < n; ++v) {
      double sz = 1.0;
      for (int f : legs[v]) sz *= (double)rsup[f] * rsup[f];
      total += sz;
    }
    if (total > 2.0 * (double)kMaxElems) {
      tnbp::set_error("the norm network is too large to contract exactly");
      return TN_EINVAL;
    }
  }
  std::vector<Tensor> net;
  for (int v = 0; v < n; ++v) {
    const int d = (int)legs[v].size();
    int64_t len = 1;
    for (int j = 0; j < d; ++j) len *= chi;
    std::vector<float> buf(4 * (size_t)len);
    st = tn_get_gamma(h, v, buf.data(), buf.size());
    if (st) return st;
    std::vector<int64_t> r(d);
    int64_t sub = 1;
    for (int j = 0; j < d; ++j) { r[j] = rsup[legs[v][j]]; sub *= r[j]; }
    // T[p][l..] = Gamma[p][l..] prod_j lambda_j[l_j]^1/2 on the supports
    std::vector<cplx> t(2 * (size_t)sub);
    std::vector<int64_t> idx(d, 0);
    for (int64_t s = 0; s < sub; ++s) {
      int64_t full = 0;
      double w = 1.0;
      for (int j = 0; j < d; ++j) {
        full = full * chi + idx[j];
        w *= std::sqrt(lam[(size_t)legs[v][j] * chi + idx[j]]);
      }
      for (int p = 0; p < 2; ++p) {
        const int64_t o = 2 * ((int64_t)p * len + full);
        t[(size_t)p * sub + s] = w * cplx(buf[o], buf[o + 1]);
      }
      for (int j = d - 1; j >= 0; --j) {
        if (++idx[j] < r[j]) break;
        idx[j] = 0;
      }
    }
    Tensor D;
    for (int j = 0; j < d; ++j) {
      const int f = legs[v][j];
      D.lab.push_back(f == e ? (edges[2 * f] == v ? m : m + 1) : f);
      D.dim.push_back(r[j] * r[j]);
    }
    int64_t dsz = 1;
    for (int64_t x : D.dim) dsz *= x;
    if (dsz > kMaxElems) {
      tnbp::set_error("a site's double-layer tensor is too large to contract exactly");
      return TN_EINVAL;
    }
    D.a.assign(dsz, cplx(0.0, 0.0));
    // D[(l_1 l_1') .. (l_d l_d')] = sum_p T[p, l..] conj(T[p, l'..])
    std::vector<int64_t> li(d, 0), lj(d, 0);
    for (int64_t s1 = 0; s1 < sub; ++s1) {
      std::fill(lj.begin(), lj.end(), 0);
      for (int64_t s2 = 0; s2 < sub; ++s2) {
        const cplx val = t[s1] * std::conj(t[s2]) + t[sub + s1] * std::conj(t[sub + s2]);
        int64_t o = 0;
        for (int j = 0; j < d; ++j) o = o * (r[j] * r[j]) + li[j] * r[j] + lj[j];
        D.a[o] = val;
        for (int j = d - 1; j >= 0; --j) {
          if (++lj[j] < r[j]) break;
          lj[j] = 0;
        }
      }
      for (int j = d - 1; j >= 0; --j) {
        if (++li[j] < r[j]) break;
        li[j] = 0;
      }
    }
    net.push_back(std::move(D));
  }
  // greedy pairwise contraction
  while (net.size() > 1) {
    int bi = -1, bj = -1;
    int64_t best = -1;
    for (int i = 0; i < (int)net.size(); ++i)
      for (int j = i + 1; j < (int)net.size(); ++j) {
        if (!shares(net[i], net[j])) continue;
        const int64_t s = result_size(net[i], net[j]);
        if (best < 0 || s < best) { best = s; bi = i; bj = j; }
      }
    if (bi < 0) {  // disconnected: join the two smallest by an outer product
      std::vector<int> o(net.size());
      std::iota(o.begin(), o.end(), 0);
      std::sort(o.begin(), o.end(), [&](int a, int b) { return net[a].size() < net[b].size(); });
      bi = std::min(o[0], o[1]);
      bj = std::max(o[0], o[1]);
      best = net[bi].size() * net[bj].size();
    }
    if (best > kMaxElems) {
      tnbp::set_error("the cut norm network is too large to contract exactly (an intermediate "
                      "above 2^26 elements)");
      return TN_EINVAL;
    }
    Tensor c = contract(net[bi], net[bj]);
    net.erase(net.begin() + bj);
    net[bi] = std::move(c);
  }
  // E[(u side), (w side)]
  Tensor E = net[0];
  if (E.lab.size() != 2) { tnbp::set_error("the edge environment lost its cut indices"); return TN_EINVAL; }
  if (E.lab[0] != m) E = permute(E, {1, 0});
  const int64_t ru = E.dim[0], rw = E.dim[1];
  // the host Jacobi on E^H E is cubic in its size: chi up to 32 on the cut edge
  if (rw > 1024) {
    tnbp::set_error("edge environment with more than 1024 columns (the cut bond's index on the "
                    "edge's second endpoint, ket x bra)");
    return TN_EINVAL;
  }
  std::vector<cplx> hm((size_t)rw * rw, cplx(0.0, 0.0));  // E^H E
  for (int64_t i = 0; i < rw; ++i)
    for (int64_t j = i; j < rw; ++j) {
      cplx s(0.0, 0.0);
      for (int64_t k = 0; k < ru; ++k) s += std::conj(E.a[k * rw + i]) * E.a[k * rw + j];
      hm[i * rw + j] = s;
      hm[j * rw + i] = std::conj(s);
    }
  std::vector<double> ev = hermitian_eigenvalues(hm, (int)rw);
  std::sort(ev.begin(), ev.end(), std::greater<double>());
  double tot = 0.0;
  for (double x : ev) tot += std::max(x, 0.0);
  if (!(tot > 0.0) || !std::isfinite(tot)) {
    tnbp::set_error("the edge environment vanishes or is not finite");
    return TN_ENUMERIC;
  }
  *error = 1.0 - std::sqrt(std::max(ev[0], 0.0) / tot);
  if (n_sv) *n_sv = (int32_t)rw;
  if (sv_out)
    for (int i = 0; i < sv_capacity && i < (int)rw; ++i) sv_out[i] = std::sqrt(std::max(ev[i], 0.0));
  return TN_OK;
}
