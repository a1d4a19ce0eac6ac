// Oracle for the sliding super point method (SRE/RSRA detection + SLE/SLEA estimation)
// of "Memory efficient distributed sliding super point cardinality estimation by GPU".
//
// TEST INFRASTRUCTURE ONLY. This is a plain, slow, single-threaded CPU restatement of
// what the paper computes, written to be checked against the paper by eye. Only the
// tests, the smoke check and the benchmark's CPU-baseline leg load it; the library
// never does, and the two share no code.
//
// Encoding is the paper's own (Section 3.2): every cell ("short integer") holds an
// unsigned 16-bit distance, initialised to 65535, incremented by one at the start of
// each new slice and set to 0 when an opposite host maps to it. In window W(t,k) a
// cell is active iff its distance is < k.
//
// Readings of points the paper leaves open (each is listed, with its reason, in the
// design notes):
//  * increment saturates at 65535;
//  * merge keeps the smaller distance (the larger "age-stamp"), so that merged
//    estimators describe the union of the routers' traffic;
//  * the union SLE of a host takes, per cell, the largest distance over its r' SLEs,
//    one from each row i of SLEA (so a cell counts only if active in every row);
//  * in the tuple checks, B(i) = he_0 XOR he_i, and the overlap test of a new row i
//    compares B(i-1) >> delta with the low q-delta bits of B(i);
//  * the delta low bits of aip that no B(i) carries are enumerated, and a host is kept
//    only if its r estimators are exactly the tuple's;
//  * hash functions: multiply-add-shift with keys drawn from SplitMix64(seed); RHFG[0]
//    may instead be simple tabulation (the family Section 3.3 cites for it): four tables of
//    256 32-bit entries, one per address byte, XORed, entries drawn from SplitMix64 after
//    the keys (top 32 bits of each output);
//  * LSB(0) = 32;
//  * a host is reported when its corrected weight w^ reaches
//    w_theta = eta' * (1 - exp(-theta/eta')), which is est >= theta in exact arithmetic;
//  * w^ < 0 is clamped to 0; w^ > eta'-1, or a product of setting factors >= 1,
//    is "saturated" and clamped to eta'-1.
//
// Parity: every function here is pinned by tests (paper examples, closed forms,
// invariants, brute force) as described beside each one.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr uint16_t kInf = 65535;  // initial value of every short integer (Section 3.2)

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): one 64-bit output per call.
uint64_t splitmix64_next(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ULL;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

struct Key {
  uint64_t a;  // odd multiplier
  uint64_t b;  // additive term
};

// Multiply-add-shift hash (Dietzfelbinger 1996): the top m bits of (a*x + b) mod 2^64.
uint32_t hash_top(const Key& key, uint32_t x, unsigned m) {
  if (m == 0) return 0;
  uint64_t v = key.a * (uint64_t)x + key.b;
  return (uint32_t)(v >> (64 - m));
}

// LSB(i): index of the lowest '1' bit of i (Definition 3); LSB(0) is taken as 32.
uint32_t lsb(uint32_t x) {
  if (x == 0) return 32;
  uint32_t i = 0;
  while (((x >> i) & 1u) == 0) ++i;
  return i;
}

unsigned log2_exact(uint64_t v) {
  unsigned m = 0;
  while ((1ULL << m) < v) ++m;
  return m;
}

}  // namespace

extern "C" {

// Parameters, mirroring the paper's symbols.
struct orc_params {
  uint32_t r, q, delta, eta;        // RSRA: r rows of 2^q SREs, RHFG shift delta, eta cells per SRE
  uint32_t r2, q2, delta2, eta2;    // SLEA: r' rows of 2^q' SLEs, offset delta', eta' cells per SLE
  uint32_t k, theta;                // window length in slices, super point threshold
  uint32_t rhfg_hash;               // RHFG[0]: 0 multiply-add-shift, 1 simple tabulation
  uint32_t pad;
  uint64_t seed;                    // all hash keys derive from it
};

struct orc_derived {
  uint32_t delta;     // delta after derivation
  uint32_t tau;       // Eq. 1
  uint32_t hot_min;   // ceil(eta * rho)
  uint32_t pad;
  uint64_t row_len2;  // 2^q' * delta' + eta' - delta' cells per SLEA row (Section 4)
  double rho;         // 0.99 * (1 - e^(-1/3))
  double w_theta;     // eta' * (1 - exp(-theta/eta'))
};

enum { ORC_OK = 0, ORC_ERR_PARAM = -1, ORC_ERR_MISMATCH = -4 };
enum { ORC_SUPER = 1, ORC_SATURATED = 2 };

}  // extern "C"

namespace {

struct Oracle {
  orc_params p;
  orc_derived d;
  unsigned lg_eta, lg_eta2;
  Key H1, H2, H3, R0;
  std::vector<Key> LH;
  uint32_t tab[4][256];  // RHFG[0] tabulation tables (rhfg_hash = 1)
  std::vector<uint16_t> rsra;  // [r][2^q][eta]
  std::vector<uint16_t> slea;  // [r'][row_len2]
  uint64_t slice = 0;          // index t of the slice being scanned
  bool track_exact = false;
  // distinct (aip,bip) pairs of the last k slices, oldest first (Definition 1 ground truth)
  std::vector<std::vector<uint64_t>> window_pairs;

  size_t sre_cell(uint32_t row, uint32_t col, uint32_t c) const {
    return ((size_t)row * ((size_t)1 << p.q) + col) * p.eta + c;
  }
  size_t sle_cell(uint32_t row, uint64_t pos) const { return (size_t)row * d.row_len2 + pos; }

  // RHFG[0]: a random hash of aip onto [0, 2^q) (Section 3.3).
  uint32_t rhfg0(uint32_t aip) const {
    if (p.rhfg_hash == 0) return hash_top(R0, aip, p.q);
    uint32_t v = 0;
    for (int j = 0; j < 4; ++j) v ^= tab[j][(aip >> (8 * j)) & 0xFFu];
    return p.q == 0 ? 0u : v >> (32 - p.q);
  }
  // RHFG[i] for 1 <= i <= r-1, Eq. 6: ((aip >> i*delta) XOR RHFG[0](aip)) mod 2^q.
  uint32_t rhfg(uint32_t i, uint32_t aip) const {
    if (i == 0) return rhfg0(aip);
    uint64_t shifted = (uint64_t)aip >> ((uint64_t)i * p.delta);
    uint64_t mask = (1ULL << p.q) - 1;
    return (uint32_t)((shifted ^ rhfg0(aip)) & mask);
  }
  uint32_t h1(uint32_t bip) const { return hash_top(H1, bip, 32); }
  uint32_t h2(uint32_t bip) const { return hash_top(H2, bip, lg_eta); }
  uint32_t h3(uint32_t bip) const { return hash_top(H3, bip, lg_eta2); }
  uint32_t lh(uint32_t i, uint32_t aip) const { return hash_top(LH[i], aip, p.q2); }

  // Algorithm 3: update RSRA with one IP pair.
  void update_rsra(uint32_t aip, uint32_t bip) {
    uint32_t hbip = h1(bip);
    if (lsb(hbip) < d.tau) return;
    uint32_t dr = h2(bip);
    for (uint32_t i = 0; i < p.r; ++i) {
      uint32_t col = rhfg(i, aip);
      rsra[sre_cell(i, col, dr)] = 0;
    }
  }

  // Algorithm 6: SLEA scans one IP pair.
  void update_slea(uint32_t aip, uint32_t bip) {
    uint32_t s = h3(bip);
    for (uint32_t i = 0; i < p.r2; ++i) {
      uint64_t j = lh(i, aip);
      slea[sle_cell(i, j * p.delta2 + s)] = 0;
    }
  }

  // |SRE|^k: number of short integers of SRE (row, col) whose value is < k (Section 3.2).
  uint32_t sre_weight(uint32_t row, uint32_t col) const {
    uint32_t w = 0;
    for (uint32_t c = 0; c < p.eta; ++c)
      if (rsra[sre_cell(row, col, c)] < p.k) ++w;
    return w;
  }
  // Hot sliding rough estimator: weight no less than eta * rho (Section 3.3).
  bool hot(uint32_t row, uint32_t col) const { return sre_weight(row, col) >= d.hot_min; }

  // Number of short integers of SLEA row i whose value is < k; SF(i,k) = this / row length.
  uint64_t row_count(uint32_t row) const {
    uint64_t c = 0;
    for (uint64_t pos = 0; pos < d.row_len2; ++pos)
      if (slea[sle_cell(row, pos)] < p.k) ++c;
    return c;
  }
};

int derive(const orc_params& in, orc_params& p, orc_derived& d) {
  p = in;
  if (p.r < 3 || p.r > 16) return ORC_ERR_PARAM;          // tuple growth starts with rows 0..2
  if (p.q < 5 || p.q > 26) return ORC_ERR_PARAM;
  if (p.delta == 0) p.delta = (32 - p.q + (p.r - 2) - 1) / (p.r - 2);  // ceil((32-q)/(r-2))
  if (p.delta == 0 || p.delta >= p.q) return ORC_ERR_PARAM;            // delta < q (Eq. 6)
  if ((uint64_t)(p.r - 2) * p.delta + p.q < 32) return ORC_ERR_PARAM;   // (r-2)*delta + q >= 32
  if ((uint64_t)(p.r - 1) * p.delta + p.q > 64) return ORC_ERR_PARAM;
  if (p.eta < 2 || p.eta > 64 || (p.eta & (p.eta - 1))) return ORC_ERR_PARAM;
  if (p.r2 < 1 || p.r2 > 16 || p.q2 > 24) return ORC_ERR_PARAM;
  if (p.eta2 < 2 || p.eta2 > (1u << 16) || (p.eta2 & (p.eta2 - 1))) return ORC_ERR_PARAM;
  if (p.delta2 < 1 || p.delta2 > p.eta2) return ORC_ERR_PARAM;
  if (p.k < 1 || p.k >= kInf) return ORC_ERR_PARAM;
  if (p.theta < 1) return ORC_ERR_PARAM;
  if (p.rhfg_hash > 1) return ORC_ERR_PARAM;
  d = orc_derived{};
  d.delta = p.delta;
  // Eq. 1: tau = ceil(log2(theta/eta)), taken as the smallest tau >= 0 with eta*2^tau >= theta.
  uint32_t tau = 0;
  while (((uint64_t)p.eta << tau) < p.theta) ++tau;
  d.tau = tau;
  d.rho = 0.99 * (1.0 - std::exp(-1.0 / 3.0));
  d.hot_min = (uint32_t)std::ceil((double)p.eta * d.rho);
  d.row_len2 = ((uint64_t)1 << p.q2) * p.delta2 + p.eta2 - p.delta2;
  d.w_theta = (double)p.eta2 * (-std::expm1(-(double)p.theta / (double)p.eta2));
  return ORC_OK;
}

// Algorithm 8 plus Eq. 11-12 for one host.
void estimate_one(const Oracle& o, const std::vector<uint64_t>& counts, uint32_t aip, double* w_out,
                  double* est_out, uint32_t* u_out, uint8_t* flags_out, uint32_t* hist_out) {
  const orc_params& p = o.p;
  // Union SLE: per cell, the largest distance over the host's r' SLEs.
  std::vector<uint16_t> usle(p.eta2);
  uint64_t j0 = o.lh(0, aip);
  for (uint32_t z = 0; z < p.eta2; ++z) usle[z] = o.slea[o.sle_cell(0, j0 * p.delta2 + z)];
  for (uint32_t i = 1; i < p.r2; ++i) {
    uint64_t j = o.lh(i, aip);
    for (uint32_t z = 0; z < p.eta2; ++z) {
      uint16_t v = o.slea[o.sle_cell(i, j * p.delta2 + z)];
      if (usle[z] < v) usle[z] = v;
    }
  }
  // |USLE|^k and its per-distance histogram.
  uint32_t U = 0;
  for (uint32_t z = 0; z < p.eta2; ++z) {
    if (usle[z] < p.k) {
      ++U;
      if (hist_out) hist_out[usle[z]] += 1;
    }
  }
  // Product of the row setting factors SF(i,k), Definition 4, multiplied in row order.
  double P = 1.0;
  for (uint32_t i = 0; i < p.r2; ++i) P = P * ((double)counts[i] / (double)o.d.row_len2);
  const double eta2 = (double)p.eta2;
  uint8_t flags = 0;
  double w;
  if (P >= 1.0) {
    w = eta2 - 1.0;
    flags |= ORC_SATURATED;
  } else {
    // Eq. 12: corrected weight.
    double num = (double)U - eta2 * P;
    double den = 1.0 - P;
    w = num / den;
    if (w < 0.0) w = 0.0;
    if (!(w <= eta2 - 1.0)) {
      w = eta2 - 1.0;
      flags |= ORC_SATURATED;
    }
  }
  // Eq. 8/9: linear-counting estimate from the corrected weight.
  double est = -eta2 * std::log((eta2 - w) / eta2);
  if (w >= o.d.w_theta) flags |= ORC_SUPER;
  *w_out = w;
  *est_out = est;
  *u_out = U;
  *flags_out = flags;
}

}  // namespace

extern "C" {

int orc_derive(const orc_params* in, orc_params* out, orc_derived* d) {
  orc_params p;
  orc_derived dd;
  int rc = derive(*in, p, dd);
  if (rc) return rc;
  if (out) *out = p;
  if (d) *d = dd;
  return ORC_OK;
}

uint64_t orc_splitmix64(uint64_t* state) { return splitmix64_next(*state); }
uint32_t orc_lsb(uint32_t x) { return lsb(x); }

int orc_create(const orc_params* in, int track_exact, void** out) {
  Oracle* o = new Oracle();
  int rc = derive(*in, o->p, o->d);
  if (rc) {
    delete o;
    return rc;
  }
  o->lg_eta = log2_exact(o->p.eta);
  o->lg_eta2 = log2_exact(o->p.eta2);
  // Keys in a fixed order: H1, H2, H3, RHFG[0], LH_0 .. LH_{r'-1}; each takes a, then b.
  uint64_t s = o->p.seed;
  auto next_key = [&s]() {
    Key k;
    k.a = splitmix64_next(s) | 1ULL;
    k.b = splitmix64_next(s);
    return k;
  };
  o->H1 = next_key();
  o->H2 = next_key();
  o->H3 = next_key();
  o->R0 = next_key();
  for (uint32_t i = 0; i < o->p.r2; ++i) o->LH.push_back(next_key());
  for (int j = 0; j < 4; ++j)
    for (int v = 0; v < 256; ++v) o->tab[j][v] = (uint32_t)(splitmix64_next(s) >> 32);
  o->rsra.assign((size_t)o->p.r * ((size_t)1 << o->p.q) * o->p.eta, kInf);
  o->slea.assign((size_t)o->p.r2 * o->d.row_len2, kInf);
  o->slice = 0;
  o->track_exact = track_exact != 0;
  if (o->track_exact) o->window_pairs.assign(1, {});
  *out = o;
  return ORC_OK;
}

void orc_destroy(void* h) { delete (Oracle*)h; }

// Hash functions, exposed for tests. which: 0=H1 (32 bits), 1=H2, 2=H3, 3=RHFG[0], 4+i=LH_i.
uint32_t orc_hash(void* h, int which, uint32_t x) {
  const Oracle& o = *(Oracle*)h;
  if (which == 0) return o.h1(x);
  if (which == 1) return o.h2(x);
  if (which == 2) return o.h3(x);
  if (which == 3) return o.rhfg0(x);
  return o.lh((uint32_t)(which - 4), x);
}
uint32_t orc_rhfg(void* h, uint32_t i, uint32_t aip) { return ((Oracle*)h)->rhfg(i, aip); }
void orc_keys(void* h, uint64_t* out) {  // (a,b) pairs in key order
  const Oracle& o = *(Oracle*)h;
  size_t n = 0;
  for (const Key* k : {&o.H1, &o.H2, &o.H3, &o.R0}) { out[n++] = k->a; out[n++] = k->b; }
  for (const Key& k : o.LH) { out[n++] = k.a; out[n++] = k.b; }
}

uint64_t orc_slice(void* h) { return ((Oracle*)h)->slice; }

// Scan the IP pairs of the current slice: pairs[2*n] = {aip_0, bip_0, aip_1, bip_1, ...}.
void orc_scan(void* h, const uint32_t* pairs, uint64_t n) {
  Oracle& o = *(Oracle*)h;
  for (uint64_t x = 0; x < n; ++x) {
    uint32_t aip = pairs[2 * x], bip = pairs[2 * x + 1];
    o.update_rsra(aip, bip);
    o.update_slea(aip, bip);
  }
  if (o.track_exact) {
    std::vector<uint64_t>& cur = o.window_pairs.back();
    for (uint64_t x = 0; x < n; ++x) cur.push_back(((uint64_t)pairs[2 * x] << 32) | pairs[2 * x + 1]);
    std::sort(cur.begin(), cur.end());
    cur.erase(std::unique(cur.begin(), cur.end()), cur.end());
  }
}

// Slice updating (Section 3.2): every short integer grows by one before the next slice.
void orc_advance(void* h) {
  Oracle& o = *(Oracle*)h;
  for (uint16_t& v : o.rsra) if (v != kInf) v = (uint16_t)(v + 1);
  for (uint16_t& v : o.slea) if (v != kInf) v = (uint16_t)(v + 1);
  o.slice += 1;
  if (o.track_exact) {
    o.window_pairs.push_back({});
    while (o.window_pairs.size() > o.p.k) o.window_pairs.erase(o.window_pairs.begin());
  }
}

// Raw distances, layout [r][2^q][eta] and [r'][row_len2].
void orc_raw(void* h, uint16_t* sre, uint16_t* sle) {
  const Oracle& o = *(Oracle*)h;
  if (sre) std::memcpy(sre, o.rsra.data(), o.rsra.size() * 2);
  if (sle) std::memcpy(sle, o.slea.data(), o.slea.size() * 2);
}
void orc_set_raw(void* h, const uint16_t* sre, const uint16_t* sle) {
  Oracle& o = *(Oracle*)h;
  if (sre) std::memcpy(o.rsra.data(), sre, o.rsra.size() * 2);
  if (sle) std::memcpy(o.slea.data(), sle, o.slea.size() * 2);
}

// Canonical state for comparisons: the distance where it is < k (the cell's age), else 255.
void orc_canonical(void* h, uint8_t* sre, uint8_t* sle) {
  const Oracle& o = *(Oracle*)h;
  for (size_t x = 0; x < o.rsra.size(); ++x) sre[x] = o.rsra[x] < o.p.k ? (uint8_t)o.rsra[x] : 255;
  for (size_t x = 0; x < o.slea.size(); ++x) sle[x] = o.slea[x] < o.p.k ? (uint8_t)o.slea[x] : 255;
}

// Hot flag of every SRE, layout [r][2^q].
void orc_hot(void* h, uint8_t* out) {
  const Oracle& o = *(Oracle*)h;
  for (uint32_t i = 0; i < o.p.r; ++i)
    for (uint32_t j = 0; j < (1u << o.p.q); ++j) out[(size_t)i * (1u << o.p.q) + j] = o.hot(i, j) ? 1 : 0;
}

// Active cells per SLEA row (numerators of SF(i,k)).
void orc_row_counts(void* h, uint64_t* out) {
  const Oracle& o = *(Oracle*)h;
  for (uint32_t i = 0; i < o.p.r2; ++i) out[i] = o.row_count(i);
}

// Candidate sliding super points by growing candidate tuples (Algorithms 4 and 5) and
// regaining hosts from complete tuples. Writes up to cap hosts (ascending, unique) and
// returns how many there are.
int64_t orc_candidates(void* h, uint32_t* out, uint64_t cap) {
  const Oracle& o = *(Oracle*)h;
  const orc_params& p = o.p;
  const uint32_t mask_overlap = (1u << (p.q - p.delta)) - 1;
  // HSE(i): hot estimators of every row.
  std::vector<std::vector<uint32_t>> hse(p.r);
  for (uint32_t i = 0; i < p.r; ++i)
    for (uint32_t j = 0; j < (1u << p.q); ++j)
      if (o.hot(i, j)) hse[i].push_back(j);
  // Algorithm 4: CT_2 from HSE(0), HSE(1), HSE(2); B(1) and B(2) must overlap.
  std::vector<std::vector<uint32_t>> ctb;
  for (uint32_t he0 : hse[0])
    for (uint32_t he1 : hse[1])
      for (uint32_t he2 : hse[2]) {
        uint32_t b1 = he0 ^ he1;
        uint32_t b2 = he0 ^ he2;
        if ((b1 >> p.delta) != (b2 & mask_overlap)) continue;
        ctb.push_back({he0, he1, he2});
      }
  // Algorithm 5: extend with HSE(i), i >= 3; only B(i-1) and B(i) are tested.
  for (uint32_t i = 3; i < p.r; ++i) {
    std::vector<std::vector<uint32_t>> next;
    for (const std::vector<uint32_t>& ct : ctb)
      for (uint32_t hei : hse[i]) {
        uint32_t bprev = ct[0] ^ ct[i - 1];
        uint32_t bi = ct[0] ^ hei;
        if ((bprev >> p.delta) != (bi & mask_overlap)) continue;
        std::vector<uint32_t> grown = ct;
        grown.push_back(hei);
        next.push_back(grown);
      }
    ctb.swap(next);
  }
  // Regain hosts: B(1) holds aip bits [delta, delta+q); each later B(i) adds its top
  // delta bits at [i*delta + q - delta, i*delta + q). Bits [0, delta) are enumerated.
  std::vector<uint32_t> hosts;
  for (const std::vector<uint32_t>& ct : ctb) {
    uint64_t high = (uint64_t)(ct[0] ^ ct[1]) << p.delta;
    for (uint32_t i = 2; i < p.r; ++i) {
      uint64_t bi = ct[0] ^ ct[i];
      high |= (bi >> (p.q - p.delta)) << ((uint64_t)i * p.delta + p.q - p.delta);
    }
    for (uint64_t low = 0; low < (1ULL << p.delta); ++low) {
      uint64_t a = high | low;
      if (a >> 32) continue;  // not a 32-bit address
      uint32_t aip = (uint32_t)a;
      bool same = true;
      for (uint32_t i = 0; i < p.r; ++i)
        if (o.rhfg(i, aip) != ct[i]) same = false;
      if (same) hosts.push_back(aip);
    }
  }
  std::sort(hosts.begin(), hosts.end());
  hosts.erase(std::unique(hosts.begin(), hosts.end()), hosts.end());
  for (uint64_t x = 0; x < hosts.size() && x < cap; ++x) out[x] = hosts[x];
  return (int64_t)hosts.size();
}

// The candidate set by its definition: every 32-bit aip whose r estimators RSRA(aip)
// are all hot. Brute force over all 2^32 addresses, split over nthreads threads.
int64_t orc_candidates_brute(void* h, uint32_t* out, uint64_t cap, int nthreads) {
  const Oracle& o = *(Oracle*)h;
  const orc_params& p = o.p;
  std::vector<std::vector<uint8_t>> hot(p.r, std::vector<uint8_t>(1u << p.q));
  for (uint32_t i = 0; i < p.r; ++i)
    for (uint32_t j = 0; j < (1u << p.q); ++j) hot[i][j] = o.hot(i, j) ? 1 : 0;
  if (nthreads < 1) nthreads = 1;
  std::vector<std::vector<uint32_t>> found(nthreads);
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t) {
    pool.emplace_back([&, t]() {
      uint64_t lo = ((uint64_t)1 << 32) * t / nthreads, hi = ((uint64_t)1 << 32) * (t + 1) / nthreads;
      for (uint64_t a = lo; a < hi; ++a) {
        uint32_t aip = (uint32_t)a;
        bool all = true;
        for (uint32_t i = 0; i < p.r && all; ++i) all = hot[i][o.rhfg(i, aip)] != 0;
        if (all) found[t].push_back(aip);
      }
    });
  }
  for (std::thread& th : pool) th.join();
  std::vector<uint32_t> hosts;
  for (auto& f : found) hosts.insert(hosts.end(), f.begin(), f.end());
  std::sort(hosts.begin(), hosts.end());
  for (uint64_t x = 0; x < hosts.size() && x < cap; ++x) out[x] = hosts[x];
  return (int64_t)hosts.size();
}

// Algorithm 8 for n hosts. Outputs per host: corrected weight w^ (Eq. 12), estimate
// (Eq. 8 on w^), |USLE|^k, flags (ORC_SUPER when w^ >= w_theta, ORC_SATURATED), and
// optionally hist[n][k]: cells of the union SLE per distance 0..k-1.
void orc_estimate(void* h, const uint32_t* hosts, uint64_t n, double* w, double* est, uint32_t* U,
                  uint8_t* flags, uint32_t* hist) {
  const Oracle& o = *(Oracle*)h;
  std::vector<uint64_t> counts(o.p.r2);
  for (uint32_t i = 0; i < o.p.r2; ++i) counts[i] = o.row_count(i);
  if (hist) std::memset(hist, 0, sizeof(uint32_t) * n * o.p.k);
  for (uint64_t x = 0; x < n; ++x)
    estimate_one(o, counts, hosts[x], &w[x], &est[x], &U[x], &flags[x], hist ? hist + x * o.p.k : nullptr);
}

// End-of-slice detection: candidates (Algorithms 4-5) then Algorithm 8 on each; returns
// the number of candidates; all of them are written (ascending) with their estimates and flags.
int64_t orc_detect(void* h, uint32_t* hosts, double* w, double* est, uint8_t* flags, uint64_t cap) {
  std::vector<uint32_t> all;
  int64_t n = orc_candidates(h, nullptr, 0);
  all.resize((size_t)n);
  orc_candidates(h, all.data(), all.size());
  std::vector<uint32_t> U(all.size());
  std::vector<double> ww(all.size()), ee(all.size());
  std::vector<uint8_t> ff(all.size());
  orc_estimate(h, all.data(), all.size(), ww.data(), ee.data(), U.data(), ff.data(), nullptr);
  for (uint64_t x = 0; x < all.size() && x < cap; ++x) {
    hosts[x] = all[x];
    w[x] = ww[x];
    est[x] = ee[x];
    flags[x] = ff[x];
  }
  return n;
}

// Weights |SRE_i|^k of each host's r estimators RSRA[i, RHFG[i](aip)]: out[n][r].
void orc_sre_weights(void* h, const uint32_t* hosts, uint64_t n, uint32_t* out) {
  const Oracle& o = *(Oracle*)h;
  for (uint64_t x = 0; x < n; ++x)
    for (uint32_t i = 0; i < o.p.r; ++i) out[x * o.p.r + i] = o.sre_weight(i, o.rhfg(i, hosts[x]));
}

// Merge (Algorithms 2 and 7, read as keeping the smaller distance): dst absorbs srcs.
int orc_merge(void* dst, void* const* srcs, int n) {
  Oracle& o = *(Oracle*)dst;
  for (int s = 0; s < n; ++s) {
    const Oracle& x = *(const Oracle*)srcs[s];
    if (std::memcmp(&x.p, &o.p, sizeof(orc_params)) != 0 || x.slice != o.slice) return ORC_ERR_MISMATCH;
  }
  for (int s = 0; s < n; ++s) {
    const Oracle& x = *(const Oracle*)srcs[s];
    for (size_t c = 0; c < o.rsra.size(); ++c) o.rsra[c] = std::min(o.rsra[c], x.rsra[c]);
    for (size_t c = 0; c < o.slea.size(); ++c) o.slea[c] = std::min(o.slea[c], x.slea[c]);
  }
  return ORC_OK;
}

// Exact |OH(aip,t,k)| (Definition 1) of the current window, from the recorded pairs.
int orc_exact_counts(void* h, const uint32_t* hosts, uint64_t n, uint32_t* out) {
  const Oracle& o = *(Oracle*)h;
  if (!o.track_exact) return ORC_ERR_PARAM;
  std::vector<uint64_t> all;
  for (const auto& sl : o.window_pairs) all.insert(all.end(), sl.begin(), sl.end());
  std::sort(all.begin(), all.end());
  all.erase(std::unique(all.begin(), all.end()), all.end());
  for (uint64_t x = 0; x < n; ++x) {
    uint64_t lo = (uint64_t)hosts[x] << 32;
    auto a = std::lower_bound(all.begin(), all.end(), lo);
    auto b = std::lower_bound(all.begin(), all.end(), lo + (1ULL << 32));
    out[x] = (uint32_t)(b - a);
  }
  return ORC_OK;
}

// Exact sliding super points of the current window (Definition 2): hosts with
// |OH(aip,t,k)| >= theta, ascending. Returns their number (or an error).
int64_t orc_exact_super(void* h, uint32_t theta, uint32_t* out, uint32_t* card, uint64_t cap) {
  const Oracle& o = *(Oracle*)h;
  if (!o.track_exact) return ORC_ERR_PARAM;
  std::vector<uint64_t> all;
  for (const auto& sl : o.window_pairs) all.insert(all.end(), sl.begin(), sl.end());
  std::sort(all.begin(), all.end());
  all.erase(std::unique(all.begin(), all.end()), all.end());
  int64_t found = 0;
  size_t x = 0;
  while (x < all.size()) {
    size_t y = x;
    while (y < all.size() && (all[y] >> 32) == (all[x] >> 32)) ++y;
    if (y - x >= theta) {
      if ((uint64_t)found < cap) {
        out[found] = (uint32_t)(all[x] >> 32);
        if (card) card[found] = (uint32_t)(y - x);
      }
      ++found;
    }
    x = y;
  }
  return found;
}

}  // extern "C"
