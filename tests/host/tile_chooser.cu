// Host-only driver of the launch-shape helpers in kernels.h (no CUDA calls):
// prints, for a grid of cases, the tile choose_tile picks against a model
// of occupancy (shared memory per CTA of a bucketed tile, a register cap),
// and the lanes choose_lanes picks.  tests/test_host_logic.py checks them.
#include <cstdio>

#include "../../paper_1010_2107_gb300/csrc/kernels.h"

int main() {
  const int threads_list[] = {128, 256, 384, 512};
  const int N_list[] = {16, 32, 50, 100, 256};
  const int dN_list[] = {200, 400, 1000};
  std::printf("[\n");
  bool first = true;
  for (int threads : threads_list)
    for (int N : N_list)
      for (int dN : dN_list)
        for (int reg_cap : {1, 2, 4})
          for (int ppt_req : {0, 1, 2, 4})
            for (int ppt_min : {1, 2})
              for (int small : {0, 1, 2}) {  // 2: the small policy with the dense floor
                // model: 227 KB per SM, bytes = dN (cap + 4) 4 + 8 dN
                auto occ_of = [&](int cap, int) {
                  const long bytes = (long)dN * (cap + 4) * 4 + 8L * dN;
                  if (bytes > 227L * 1024) return 0;
                  const int o = (int)((227L * 1024) / bytes);
                  return o < reg_cap ? o : reg_cap;
                };
                const gv::TileShape t =
                    gv::choose_tile(threads, N, ppt_req, ppt_min, reg_cap, occ_of, small != 0, small == 2);
                std::printf("%s{\"threads\":%d,\"N\":%d,\"dN\":%d,\"reg_cap\":%d,\"ppt_req\":%d,\"ppt_min\":%d,"
                            "\"small\":%d,\"ppt\":%d,\"cap\":%d,\"occ\":%d,\"occ_check\":%d}\n",
                            first ? "" : ",", threads, N, dN, reg_cap, ppt_req, ppt_min, small, t.ppt, t.cap, t.occ,
                            t.cap > 0 ? occ_of(t.cap, t.ppt) : -1);
                first = false;
              }
  std::printf("]\n");
  // lanes per hypercube
  std::printf("LANES");
  const unsigned long long G_list[] = {1, 64, 1024, 32768, 65536, 1048576};
  const unsigned long long nc_list[] = {2, 4, 64, 128, 4096};
  for (unsigned long long G : G_list)
    for (unsigned long long nc : nc_list)
      for (int threads : {256, 384})
        for (long ctas : {152L, 456L, 608L})
          std::printf(" %llu,%llu,%d,%ld,%d", G, nc, threads, ctas, gv::choose_lanes(G, nc, threads, ctas));
  std::printf("\n");
  return 0;
}
