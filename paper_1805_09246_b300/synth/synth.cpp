// Seeded synthetic IP-pair traffic for the sliding super point workloads.
//
// This module only makes inputs. It holds none of the estimator arithmetic; the CUDA
// library and the CPU oracle both consume its output as plain data.
//
// Model (stated in full in the design notes):
//  * a background population of n_sources hosts; host of popularity rank n (0-based)
//    has address ip(n), a bijective 32-bit mix of n, and m_n distinct destinations,
//    m_n uniform in [bg_dst_min, bg_dst_max];
//  * a background packet picks its source by Zipf(zipf_s) popularity (Walker/Vose alias
//    table) and its destination uniformly among that source's m_n destinations;
//  * n_planted super points (ranks n_sources .. n_sources+n_planted-1) each contact
//    c_p distinct uniform random destinations, c_p uniform or log-uniform in
//    [planted_min, planted_max]; each destination is sent exactly once, in a uniform
//    slice of [planted_slice_lo, planted_slice_hi) and by one router of the host's
//    router group (1..R consecutive routers);
//  * the (router, slice) stream has load_min..load_max pairs (log-uniform; at least the
//    number of planted pairs it carries); planted pairs are shuffled and placed one per
//    equal-width stratum of the stream, background pairs fill the other positions.
// Randomness: Philox4x32-10 (Salmon et al., SC'11), counter = (a, b, c, tag), key = seed,
// so every value is a pure function of its coordinates and thread count never matters.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

struct U4 {
  uint32_t v[4];
};

U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  return U4{{c0, c1, c2, c3}};
}

enum : uint32_t {
  TAG_SRC_M = 1, TAG_SRC_DST = 2, TAG_PL_CARD = 3, TAG_PL_DST = 4, TAG_PL_GROUP = 5,
  TAG_LOAD = 6, TAG_BG = 7, TAG_SHUFFLE = 8, TAG_POS = 9, TAG_IP = 10
};

// Uniform double in [0,1) from 32 random bits.
double unit(uint32_t x) { return (double)x * (1.0 / 4294967296.0); }
// Uniform integer in [0, n) by multiply-shift.
uint32_t below(uint32_t x, uint32_t n) { return (uint32_t)(((uint64_t)x * n) >> 32); }

}  // namespace

extern "C" {

struct synth_config {
  uint64_t seed;
  uint32_t n_slices;
  uint32_t n_routers;
  uint64_t load_min, load_max;         // pairs per (router, slice), log-uniform
  uint32_t n_sources;                  // background population
  uint32_t bg_dst_min, bg_dst_max;     // distinct destinations per background host
  uint32_t n_planted;                  // planted super points
  uint32_t planted_min, planted_max;   // their cardinalities
  uint32_t planted_log;                // 0: uniform integer, 1: log-uniform
  uint32_t group_min, group_max;       // routers per planted host
  uint32_t planted_slice_lo, planted_slice_hi;
  uint32_t pad;
  double zipf_s;
};

}  // extern "C"

namespace {

struct Synth {
  synth_config c;
  uint32_t k0, k1;
  uint32_t ip_in, ip_out;            // keys of the address mix
  std::vector<uint32_t> alias_prob;  // threshold in 2^-32 units
  std::vector<uint32_t> alias_idx;
  std::vector<uint8_t> dst_count;    // m_n
  std::vector<uint32_t> planted_ip, planted_card;
  // planted pairs bucketed by (router, slice)
  std::vector<uint64_t> bucket_off;  // n_routers * n_slices + 1
  std::vector<uint32_t> bucket_src, bucket_dst;

  U4 rnd(uint32_t a, uint32_t b, uint32_t c2, uint32_t tag) const { return philox4x32_10(a, b, c2, tag, k0, k1); }

  // Bijective 32-bit mix of a rank: distinct ranks give distinct addresses.
  uint32_t ip_of_rank(uint32_t n) const {
    uint32_t x = n ^ ip_in;
    x ^= x >> 16; x *= 0x7FEB352Du;
    x ^= x >> 15; x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x ^ ip_out;
  }

  uint64_t load(uint32_t router, uint32_t slice) const {
    uint64_t lo = c.load_min, hi = c.load_max, n;
    if (hi <= lo) {
      n = lo;
    } else {
      double u = unit(rnd(router, slice, 0, TAG_LOAD).v[0]);
      n = (uint64_t)std::floor(std::exp(std::log((double)lo) + u * (std::log((double)hi) - std::log((double)lo))));
      n = std::min(std::max(n, lo), hi);
    }
    uint64_t b = (uint64_t)router * c.n_slices + slice;
    uint64_t planted = bucket_off[b + 1] - bucket_off[b];
    return std::max(n, planted);
  }

  void background(uint64_t i, uint32_t router, uint32_t slice, uint32_t* out) const {
    U4 r = rnd((uint32_t)i, (uint32_t)(i >> 32) ^ (slice << 8), router, TAG_BG);
    uint32_t col = below(r.v[0], c.n_sources);
    uint32_t n = r.v[1] < alias_prob[col] ? col : alias_idx[col];
    uint32_t j = below(r.v[2], dst_count[n]);
    out[0] = ip_of_rank(n);
    out[1] = rnd(n, j, 0, TAG_SRC_DST).v[0];
  }
};

void build_alias(Synth& s) {
  // Vose's alias method over weights (n+1)^-s, n in [0, N).
  const uint32_t N = s.c.n_sources;
  std::vector<double> w(N);
  double sum = 0;
  for (uint32_t n = 0; n < N; ++n) sum += (w[n] = std::pow((double)n + 1.0, -s.c.zipf_s));
  for (uint32_t n = 0; n < N; ++n) w[n] = w[n] * N / sum;
  std::vector<uint32_t> small, large;
  for (uint32_t n = 0; n < N; ++n) (w[n] < 1.0 ? small : large).push_back(n);
  s.alias_prob.assign(N, 0xFFFFFFFFu);
  s.alias_idx.resize(N);
  for (uint32_t n = 0; n < N; ++n) s.alias_idx[n] = n;
  while (!small.empty() && !large.empty()) {
    uint32_t l = small.back(); small.pop_back();
    uint32_t g = large.back(); large.pop_back();
    s.alias_prob[l] = (uint32_t)std::min(4294967295.0, w[l] * 4294967296.0);
    s.alias_idx[l] = g;
    w[g] = (w[g] + w[l]) - 1.0;
    (w[g] < 1.0 ? small : large).push_back(g);
  }
}

}  // namespace

extern "C" {

int synth_create(const synth_config* cfg, void** out) {
  if (!cfg || cfg->n_slices == 0 || cfg->n_routers == 0 || cfg->n_sources == 0 || cfg->load_min == 0 ||
      cfg->bg_dst_min == 0 || cfg->bg_dst_max < cfg->bg_dst_min || cfg->bg_dst_max > 255 ||
      cfg->planted_slice_hi > cfg->n_slices || cfg->planted_slice_lo >= cfg->planted_slice_hi ||
      (cfg->n_planted && (cfg->planted_min == 0 || cfg->planted_max < cfg->planted_min)) ||
      cfg->group_min == 0 || cfg->group_max < cfg->group_min || cfg->group_max > cfg->n_routers)
    return -1;
  Synth* s = new Synth();
  s->c = *cfg;
  s->k0 = (uint32_t)cfg->seed;
  s->k1 = (uint32_t)(cfg->seed >> 32);
  U4 ipk = s->rnd(0, 0, 0, TAG_IP);
  s->ip_in = ipk.v[0];
  s->ip_out = ipk.v[1];
  build_alias(*s);
  s->dst_count.resize(cfg->n_sources);
  const uint32_t span = cfg->bg_dst_max - cfg->bg_dst_min + 1;
  for (uint32_t n = 0; n < cfg->n_sources; ++n)
    s->dst_count[n] = (uint8_t)(cfg->bg_dst_min + below(s->rnd(n, 0, 0, TAG_SRC_M).v[0], span));
  // Planted super points.
  const uint32_t R = cfg->n_routers, T = cfg->n_slices;
  std::vector<uint64_t> counts((size_t)R * T + 1, 0);
  struct Ent { uint32_t p, dst, bucket; };
  std::vector<Ent> ents;
  for (uint32_t p = 0; p < cfg->n_planted; ++p) {
    U4 r = s->rnd(p, 0, 0, TAG_PL_CARD);
    double lo = cfg->planted_min, hi = cfg->planted_max;
    uint32_t card;
    if (cfg->planted_log)
      card = (uint32_t)std::floor(std::exp(std::log(lo) + unit(r.v[0]) * (std::log(hi) - std::log(lo))));
    else
      card = cfg->planted_min + below(r.v[0], cfg->planted_max - cfg->planted_min + 1);
    card = std::min(std::max(card, cfg->planted_min), cfg->planted_max);
    s->planted_ip.push_back(s->ip_of_rank(cfg->n_sources + p));
    s->planted_card.push_back(card);
    U4 g = s->rnd(p, 0, 0, TAG_PL_GROUP);
    uint32_t gsize = cfg->group_min + below(g.v[0], cfg->group_max - cfg->group_min + 1);
    uint32_t gbase = below(g.v[1], R);
    for (uint32_t j = 0; j < card; ++j) {
      U4 d = s->rnd(p, j, 0, TAG_PL_DST);
      uint32_t slice = cfg->planted_slice_lo + below(d.v[1], cfg->planted_slice_hi - cfg->planted_slice_lo);
      uint32_t router = (gbase + below(d.v[2], gsize)) % R;
      uint32_t b = router * T + slice;
      ents.push_back(Ent{p, d.v[0], b});
      counts[b + 1] += 1;
    }
  }
  for (size_t b = 1; b < counts.size(); ++b) counts[b] += counts[b - 1];
  s->bucket_off = counts;
  s->bucket_src.resize(ents.size());
  s->bucket_dst.resize(ents.size());
  std::vector<uint64_t> fill(counts.begin(), counts.end() - 1);
  for (const Ent& e : ents) {
    uint64_t at = fill[e.bucket]++;
    s->bucket_src[at] = s->planted_ip[e.p];
    s->bucket_dst[at] = e.dst;
  }
  *out = s;
  return 0;
}

void synth_destroy(void* h) { delete (Synth*)h; }

uint64_t synth_slice_len(void* h, uint32_t router, uint32_t slice) { return ((Synth*)h)->load(router, slice); }

uint64_t synth_planted_in(void* h, uint32_t router, uint32_t slice) {
  const Synth& s = *(Synth*)h;
  uint64_t b = (uint64_t)router * s.c.n_slices + slice;
  return s.bucket_off[b + 1] - s.bucket_off[b];
}

// Planted super point addresses and their total cardinalities (over all slices/routers).
void synth_planted(void* h, uint32_t* ip, uint32_t* card) {
  const Synth& s = *(Synth*)h;
  for (size_t p = 0; p < s.planted_ip.size(); ++p) {
    if (ip) ip[p] = s.planted_ip[p];
    if (card) card[p] = s.planted_card[p];
  }
}

uint32_t synth_source_ip(void* h, uint32_t rank) { return ((Synth*)h)->ip_of_rank(rank); }

// Writes the (router, slice) stream, synth_slice_len() pairs, as {src, dst} u32 pairs.
int synth_fill(void* h, uint32_t router, uint32_t slice, uint32_t* out, uint64_t cap, int nthreads) {
  const Synth& s = *(Synth*)h;
  if (router >= s.c.n_routers || slice >= s.c.n_slices) return -1;
  const uint64_t len = s.load(router, slice);
  if (cap < len) return -2;
  const uint64_t b = (uint64_t)router * s.c.n_slices + slice;
  const uint64_t m = s.bucket_off[b + 1] - s.bucket_off[b];
  // Planted pairs of this stream, shuffled (Fisher-Yates) ...
  std::vector<uint32_t> order(m);
  for (uint64_t e = 0; e < m; ++e) order[e] = (uint32_t)e;
  for (uint64_t e = m; e > 1; --e) {
    uint32_t j = below(s.rnd((uint32_t)e, slice, router, TAG_SHUFFLE).v[0], (uint32_t)e);
    std::swap(order[e - 1], order[j]);
  }
  // ... and placed one per stratum [floor(e*len/m), floor((e+1)*len/m)).
  std::vector<uint64_t> pos(m);
  for (uint64_t e = 0; e < m; ++e) {
    uint64_t lo = e * len / m, hi = (e + 1) * len / m;
    pos[e] = lo + below(s.rnd((uint32_t)e, slice, router, TAG_POS).v[0], (uint32_t)(hi - lo));
  }
  if (nthreads < 1) nthreads = 1;
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t) {
    pool.emplace_back([&, t]() {
      uint64_t lo = len * t / nthreads, hi = len * (t + 1) / nthreads;
      uint64_t e = std::lower_bound(pos.begin(), pos.end(), lo) - pos.begin();
      for (uint64_t i = lo; i < hi; ++i) {
        if (e < m && pos[e] == i) {
          uint64_t at = s.bucket_off[b] + order[e];
          out[2 * i] = s.bucket_src[at];
          out[2 * i + 1] = s.bucket_dst[at];
          ++e;
        } else {
          s.background(i - e, router, slice, out + 2 * i);
        }
      }
    });
  }
  for (std::thread& th : pool) th.join();
  return 0;
}

// Philox4x32-10 block, exposed so tests can check it against the published answers.
void synth_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  U4 r = philox4x32_10(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1]);
  std::memcpy(out, r.v, 16);
}

}  // extern "C"
