// tune.cu -- the tuning cache of libmw: keys and a JSON-lines file (host only).
//
// A key names what a tuning depends on: the sorted multiset of (band limit,
// spin) over the plan's maps, the precision, the Wigner recursion, the
// real-signal flag and the device.  The cache file holds one JSON object per
// line,
//   {"key": "<key>", "chunk": 512, "groups": 2, "tn_threads": 256, "ms": 62.512}
// and a store replaces the line of its key (or appends one) by writing the
// whole file to a temporary name and renaming it into place.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unistd.h>
#include <utility>
#include <vector>

#include "internal.h"

namespace {

// value of the integer field `name` in a cache line, or `fallback`
int field_int(const std::string& line, const char* name, int fallback) {
  const std::string pat = std::string("\"") + name + "\":";
  const size_t at = line.find(pat);
  if (at == std::string::npos) return fallback;
  return atoi(line.c_str() + at + pat.size());
}

double field_double(const std::string& line, const char* name, double fallback) {
  const std::string pat = std::string("\"") + name + "\":";
  const size_t at = line.find(pat);
  if (at == std::string::npos) return fallback;
  return atof(line.c_str() + at + pat.size());
}

// the key of a cache line ("" if the line has none)
std::string line_key(const std::string& line) {
  const std::string pat = "\"key\": \"";
  const size_t at = line.find(pat);
  if (at == std::string::npos) return "";
  const size_t end = line.find('"', at + pat.size());
  if (end == std::string::npos) return "";
  return line.substr(at + pat.size(), end - at - pat.size());
}

bool read_lines(const char* path, std::vector<std::string>* lines) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  std::string cur;
  int c;
  while ((c = fgetc(f)) != EOF) {
    if (c == '\n') {
      if (!cur.empty()) lines->push_back(cur);
      cur.clear();
    } else {
      cur.push_back((char)c);
    }
  }
  if (!cur.empty()) lines->push_back(cur);
  fclose(f);
  return true;
}

}  // namespace

extern "C" {

mw_status mw_tune_key(int n, const int* L, const int* spins, unsigned flags, const char* device, char* key,
                      size_t len) {
  if (n < 1 || !L || !spins || !key) return MW_EINVAL;
  std::vector<std::pair<int, int>> ms(n);
  for (int b = 0; b < n; ++b) ms[b] = {L[b], spins[b]};
  std::sort(ms.begin(), ms.end());
  std::string k = "maps=";
  for (int i = 0; i < n;) {
    int j = i;
    while (j < n && ms[j] == ms[i]) ++j;
    char buf[64];
    snprintf(buf, sizeof(buf), "%s%d/%dx%d", i ? "," : "", ms[i].first, ms[i].second, j - i);
    k += buf;
    i = j;
  }
  const int prec = (int)(flags & 0xffu);
  const bool risbo = (flags & MW_FLAG_DELTA_RISBO) || prec == MW_PREC_FP64;
  char buf[64];
  snprintf(buf, sizeof(buf), ";prec=%d;delta=%s;real=%d;dev=", prec, risbo ? "risbo" : "tn",
           (flags & MW_FLAG_REAL) ? 1 : 0);
  k += buf;
  for (const char* c = device ? device : ""; *c; ++c) k.push_back((*c == '"' || *c == '\\' || *c == ';') ? '_' : *c);
  if (k.size() + 1 > len) return MW_EINVAL;
  memcpy(key, k.c_str(), k.size() + 1);
  return MW_OK;
}

mw_status mw_tune_cache_lookup(const char* path, const char* key, mw_tuning* out, int* found) {
  if (!path || !key || !out || !found) return MW_EINVAL;
  *found = 0;
  std::vector<std::string> lines;
  if (!read_lines(path, &lines)) return MW_OK;  // no cache yet
  for (const std::string& ln : lines) {
    if (line_key(ln) != key) continue;
    out->chunk = field_int(ln, "chunk", 512);
    out->groups = field_int(ln, "groups", 2);
    out->tn_threads = field_int(ln, "tn_threads", 256);
    out->ms = field_double(ln, "ms", 0.0);
    *found = 1;
  }
  return MW_OK;
}

mw_status mw_tune_cache_store(const char* path, const char* key, const mw_tuning* t) {
  if (!path || !key || !t || strchr(key, '"') || strchr(key, '\n')) return MW_EINVAL;
  std::vector<std::string> lines, kept;
  read_lines(path, &lines);
  char buf[160];
  snprintf(buf, sizeof(buf), "\"chunk\": %d, \"groups\": %d, \"tn_threads\": %d, \"ms\": %.6f}", t->chunk, t->groups,
           t->tn_threads, t->ms);
  const std::string mine = std::string("{\"key\": \"") + key + "\", " + buf;
  bool placed = false;
  for (const std::string& ln : lines) {
    if (line_key(ln) == key) {
      if (!placed) kept.push_back(mine);
      placed = true;
    } else {
      kept.push_back(ln);
    }
  }
  if (!placed) kept.push_back(mine);
  const std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid());
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return MW_EINVAL;
  bool ok = true;
  for (const std::string& ln : kept) ok = ok && fprintf(f, "%s\n", ln.c_str()) > 0;
  ok = (fclose(f) == 0) && ok;
  if (!ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return MW_EINVAL;
  }
  return MW_OK;
}

}  // extern "C"
