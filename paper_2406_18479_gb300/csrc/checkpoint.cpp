// Checkpoint files of a self-consistent loop: a one-line JSON header followed by the named
// complex arrays as raw little-endian complex128 values, in header order.
//
//   {"format": "gw-gb300-checkpoint", "version": 1, "nk": [N1, N2, N3], "nao": .., "naux": ..,
//    "ntau": .., "beta": .., "spin_factor": .., "mu": .., "iteration": ..,
//    "arrays": [{"name": "G", "count": ..}, ...]}\n<raw values>
//
// The header is written and read by this file only (a fixed layout, not a general JSON parser).
// Host memory on both sides; a loop continues from a checkpoint through gw_scgw's resume option.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gw_internal.h"

using namespace gwi;

namespace {

bool little_endian() {
  const uint16_t one = 1;
  unsigned char b;
  std::memcpy(&b, &one, 1);
  return b == 1;
}

// value following "key": in the header (numbers only)
bool find_number(const std::string& h, const char* key, double* out) {
  const std::string k = std::string("\"") + key + "\":";
  const size_t p = h.find(k);
  if (p == std::string::npos) return false;
  const char* s = h.c_str() + p + k.size();
  char* end = nullptr;
  *out = std::strtod(s, &end);
  return end != s;
}

bool valid_name(const char* n) {
  if (!n || !*n || std::strlen(n) > 64) return false;
  for (const char* c = n; *c; ++c)
    if (!((*c >= 'a' && *c <= 'z') || (*c >= 'A' && *c <= 'Z') || (*c >= '0' && *c <= '9') || *c == '_'))
      return false;
  return true;
}

}  // namespace

extern "C" {

int gw_checkpoint_write(const char* path, const gw_config* cfg, double mu, int iteration, int narrays,
                        const char* const* names, const gw_c128* const* data_host, const long long* counts) {
  if (!path || !cfg || narrays < 0 || narrays > 64 || (narrays > 0 && (!names || !data_host || !counts)))
    return fail(GW_EINVAL, "gw_checkpoint_write: bad argument");
  if (!little_endian()) return fail(GW_ENOTIMPL, "gw_checkpoint_write: little-endian hosts only");
  for (int i = 0; i < narrays; ++i)
    if (!valid_name(names[i]) || counts[i] < 0 || (counts[i] > 0 && !data_host[i]))
      return fail(GW_EINVAL, "gw_checkpoint_write: bad array %d", i);
  char buf[512];
  std::snprintf(buf, sizeof buf,
                "{\"format\": \"gw-gb300-checkpoint\", \"version\": 1, \"nk\": [%d, %d, %d], \"nao\": %d, "
                "\"naux\": %d, \"ntau\": %d, \"beta\": %.17g, \"spin_factor\": %.17g, \"mu\": %.17g, "
                "\"iteration\": %d, \"arrays\": [",
                cfg->nk[0], cfg->nk[1], cfg->nk[2], cfg->nao, cfg->naux, cfg->ntau, cfg->beta, cfg->spin_factor, mu,
                iteration);
  std::string h = buf;
  for (int i = 0; i < narrays; ++i) {
    std::snprintf(buf, sizeof buf, "%s{\"name\": \"%s\", \"count\": %lld}", i ? ", " : "", names[i], counts[i]);
    h += buf;
  }
  h += "]}\n";
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(GW_EINVAL, "gw_checkpoint_write: cannot open %s", path);
  bool ok = std::fwrite(h.data(), 1, h.size(), f) == h.size();
  for (int i = 0; ok && i < narrays; ++i)
    ok = std::fwrite(data_host[i], sizeof(gw_c128), (size_t)counts[i], f) == (size_t)counts[i];
  ok = (std::fclose(f) == 0) && ok;
  return ok ? GW_OK : fail(GW_EINVAL, "gw_checkpoint_write: write to %s failed", path);
}

int gw_checkpoint_read(const char* path, gw_config* cfg_out, double* mu, int* iteration, int narrays,
                       const char* const* names, gw_c128* const* data_host, const long long* counts) {
  if (!path || narrays < 0 || narrays > 64 || (narrays > 0 && (!names || !data_host || !counts)))
    return fail(GW_EINVAL, "gw_checkpoint_read: bad argument");
  if (!little_endian()) return fail(GW_ENOTIMPL, "gw_checkpoint_read: little-endian hosts only");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(GW_EINVAL, "gw_checkpoint_read: cannot open %s", path);
  std::string h;
  for (int c; (c = std::fgetc(f)) != EOF && c != '\n' && h.size() < 65536;) h.push_back((char)c);
  auto bad = [&](const char* why) {
    std::fclose(f);
    return fail(GW_EINVAL, "gw_checkpoint_read: %s: %s", path, why);
  };
  if (h.find("\"format\": \"gw-gb300-checkpoint\"") == std::string::npos) return bad("not a checkpoint");
  double v = 0;
  if (!find_number(h, "version", &v) || v != 1) return bad("unknown version");
  // the stored arrays, in file order
  std::vector<std::string> snames;
  std::vector<long long> scounts;
  for (size_t p = h.find("{\"name\": \""); p != std::string::npos; p = h.find("{\"name\": \"", p + 1)) {
    const size_t a = p + 10, b = h.find('"', a);
    if (b == std::string::npos) return bad("broken array list");
    const size_t q = h.find("\"count\": ", b);
    if (q == std::string::npos) return bad("broken array list");
    snames.push_back(h.substr(a, b - a));
    scounts.push_back(std::strtoll(h.c_str() + q + 9, nullptr, 10));
  }
  gw_config c{};
  double nk0 = 0, nk1 = 0, nk2 = 0, nao = 0, naux = 0, ntau = 0, beta = 0, sf = 0, m = 0, it = 0;
  const size_t pk = h.find("\"nk\": [");
  if (pk == std::string::npos || std::sscanf(h.c_str() + pk + 7, "%lf, %lf, %lf", &nk0, &nk1, &nk2) != 3 ||
      !find_number(h, "nao", &nao) || !find_number(h, "naux", &naux) || !find_number(h, "ntau", &ntau) ||
      !find_number(h, "beta", &beta) || !find_number(h, "spin_factor", &sf) || !find_number(h, "mu", &m) ||
      !find_number(h, "iteration", &it))
    return bad("incomplete header");
  c.nk[0] = (int)nk0;
  c.nk[1] = (int)nk1;
  c.nk[2] = (int)nk2;
  c.nao = (int)nao;
  c.naux = (int)naux;
  c.ntau = (int)ntau;
  c.beta = beta;
  c.spin_factor = sf;
  c.mu = m;
  // every requested array must be stored with the requested count; read them in file order
  std::vector<int> want(snames.size(), -1);
  for (int i = 0; i < narrays; ++i) {
    size_t j = 0;
    while (j < snames.size() && snames[j] != (names[i] ? names[i] : "")) ++j;
    if (j == snames.size()) return bad("a requested array is not stored");
    if (scounts[j] != counts[i]) return bad("an array's size differs");
    want[j] = i;
  }
  for (size_t j = 0; j < snames.size(); ++j) {
    if (scounts[j] < 0) return bad("negative count");
    if (want[j] >= 0) {
      if (std::fread(data_host[want[j]], sizeof(gw_c128), (size_t)scounts[j], f) != (size_t)scounts[j])
        return bad("truncated");
    } else if (std::fseek(f, (long)(scounts[j] * (long long)sizeof(gw_c128)), SEEK_CUR) != 0) {
      return bad("truncated");
    }
  }
  std::fclose(f);
  if (cfg_out) {
    const gw_config keep = *cfg_out;
    *cfg_out = c;
    cfg_out->precision = keep.precision;        // not part of the checkpoint
    cfg_out->tau_chunk = keep.tau_chunk;
    cfg_out->v_slices = keep.v_slices;
    cfg_out->v_packed = keep.v_packed;
    cfg_out->slice_pass = keep.slice_pass;
    cfg_out->tile_n = keep.tile_n;
  }
  if (mu) *mu = m;
  if (iteration) *iteration = (int)it;
  return GW_OK;
}

}  // extern "C"
