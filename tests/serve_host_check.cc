// Command-line driver for the server's host-only parts (arena, latency log),
// for tests/test_serve_host.py.  One command per input line:
//   reset S | alloc B | free OFF B | stat | log W | rec MS | pct P | mean | max
#include <cstdio>
#include <cstring>
#include <iostream>
#include <sstream>
#include <string>

#include "../paper_2605_10390_gb300/csrc/fsort_serve_host.h"

int main() {
  fsort_serve::Arena arena;
  fsort_serve::LatencyLog log;
  std::string line;
  while (std::getline(std::cin, line)) {
    std::istringstream in(line);
    std::string cmd;
    in >> cmd;
    if (cmd == "reset") {
      size_t s = 0;
      in >> s;
      arena.reset(s);
    } else if (cmd == "alloc") {
      size_t b = 0, off = 0;
      in >> b;
      if (arena.alloc(b, &off))
        std::printf("%zu\n", off);
      else
        std::printf("-1\n");
    } else if (cmd == "free") {
      size_t off = 0, b = 0;
      in >> off >> b;
      arena.release(off, b);
    } else if (cmd == "stat") {
      std::printf("%zu %zu %zu %zu\n", arena.size(), arena.used(), arena.peak(), arena.free_ranges());
    } else if (cmd == "log") {
      size_t w = 0;
      in >> w;
      log = fsort_serve::LatencyLog(w);
    } else if (cmd == "rec") {
      double ms = 0;
      in >> ms;
      log.record(ms);
    } else if (cmd == "pct") {
      double p = 0;
      in >> p;
      std::printf("%.17g\n", log.percentiles({p})[0]);
    } else if (cmd == "mean") {
      std::printf("%.17g\n", log.mean());
    } else if (cmd == "max") {
      std::printf("%.17g\n", log.max());
    } else if (!cmd.empty()) {
      std::fprintf(stderr, "unknown command %s\n", cmd.c_str());
      return 2;
    }
  }
  return 0;
}
