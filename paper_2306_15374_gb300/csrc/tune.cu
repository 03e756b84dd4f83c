// Tuning table: the configuration (stages in flight, consumer warps) each scan uses, keyed by
// operation, value width and the column's widest partition (which sets the stage size), and the
// batched encode's shape (values per pack item, fit CTAs per SM) per value width. Entries come from
// leco_tune_scan / leco_tune_batch_encode (timed candidates on real data) or from a JSON file.
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include "leco_internal.cuh"

namespace leco {

namespace {

std::mutex g_mu;
std::map<std::tuple<int, int, int>, ScanConfig> g_table;
std::map<int, EncodeConfig> g_enc;  // batched encode shape per value width

// 0: widest partition <= 8 bits, 1: <= 16, 2: <= 32, 3: wider
int width_bucket(uint32_t stage_bytes) {
  const uint64_t max_b = (uint64_t)(stage_bytes > 64 ? stage_bytes - 64 : 0) * 8 / kScanTile;
  return max_b <= 8 ? 0 : max_b <= 16 ? 1 : max_b <= 32 ? 2 : 3;
}

}  // namespace

ScanConfig scan_config_lookup(int op, int dtype, uint32_t stage_bytes) {
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(std::make_tuple(op, dtype, width_bucket(stage_bytes)));
  if (it != g_table.end()) return it->second;
  // untuned default: two stages and four consumer warps keep the CTA small (up to ~6 resident per
  // SM), which measured best or within 2% of best for both decode and filter-sum across widths
  return ScanConfig{2, 4};
}

ScanConfig scan_config_for(const ColumnView& c, int op) { return scan_config_lookup(op, c.dtype, c.stage_bytes); }

void scan_config_store(int op, int dtype, uint32_t stage_bytes, ScanConfig cfg) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_table[std::make_tuple(op, dtype, width_bucket(stage_bytes))] = cfg;
}

EncodeConfig encode_config_lookup(int dtype) {
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_enc.find(dtype);
  if (it != g_enc.end()) return it->second;
  return EncodeConfig{4096, 4};  // untuned default: the largest items, four fit CTAs per SM
}

void encode_config_store(int dtype, EncodeConfig cfg) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_enc[dtype] = cfg;
}

int tune_table_save(const char* path) {
  std::lock_guard<std::mutex> lock(g_mu);
  FILE* f = fopen(path, "w");
  if (!f) return -1;
  fprintf(f, "{\"scan_configs\": [");
  bool first = true;
  for (const auto& kv : g_table) {
    fprintf(f, "%s\n  {\"op\": %d, \"dtype\": %d, \"width_bucket\": %d, \"stages\": %u, \"consumer_warps\": %u}",
            first ? "" : ",", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
            kv.second.stages, kv.second.consumer_warps);
    first = false;
  }
  fprintf(f, "\n], \"encode_configs\": [");
  first = true;
  for (const auto& kv : g_enc) {
    fprintf(f, "%s\n  {\"dtype\": %d, \"item_values\": %u, \"fit_ctas\": %u}", first ? "" : ",", kv.first,
            kv.second.item_values, kv.second.fit_ctas);
    first = false;
  }
  fprintf(f, "\n]}\n");
  fclose(f);
  return 0;
}

// reads back what tune_table_save writes (one entry per line)
int tune_table_load(const char* path) {
  FILE* f = fopen(path, "r");
  if (!f) return -1;
  char line[512];
  int n = 0;
  std::lock_guard<std::mutex> lock(g_mu);
  while (fgets(line, sizeof(line), f)) {
    int op, dtype, wb;
    unsigned st, cw;
    unsigned iv, fc;
    const char* q = strstr(line, "{\"dtype\"");
    if (q && sscanf(q, "{\"dtype\": %d, \"item_values\": %u, \"fit_ctas\": %u}", &dtype, &iv, &fc) == 3 &&
        (iv == 1024 || iv == 2048 || iv == 4096) && fc >= 2 && fc <= 4) {
      g_enc[dtype] = EncodeConfig{iv, fc};
      n++;
      continue;
    }
    const char* p = strstr(line, "{\"op\"");
    if (!p) continue;
    if (sscanf(p, "{\"op\": %d, \"dtype\": %d, \"width_bucket\": %d, \"stages\": %u, \"consumer_warps\": %u}", &op,
               &dtype, &wb, &st, &cw) == 5 &&
        st >= 2 && st <= 8 && (cw == 4 || cw == 8)) {
      g_table[std::make_tuple(op, dtype, wb)] = ScanConfig{st, cw};
      n++;
    }
  }
  fclose(f);
  return n;
}

}  // namespace leco
