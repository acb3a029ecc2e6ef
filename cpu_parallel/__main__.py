"""Time the CPU-parallel scheme on one field: one warm-up run, then REPEATS
timed runs on all host cores; prints one JSON line (median and all times)."""
import json
import statistics
import sys
import time

import numpy as np

from . import max_threads, segment


def main(argv):
    if len(argv) != 3:
        print("usage: python -m cpu_parallel FIELD.npy REPEATS", file=sys.stderr)
        return 2
    f = np.load(argv[1])
    repeats = max(1, int(argv[2]))
    threads = max_threads()
    k = segment(f, threads)["K"]  # warm-up
    times = []
    for _ in range(repeats):
        t = time.perf_counter()
        segment(f, threads)
        times.append(time.perf_counter() - t)
    print(json.dumps({"vertices": int(f.size), "threads": threads, "K": k,
                      "median_s": statistics.median(times), "times_s": times}))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
