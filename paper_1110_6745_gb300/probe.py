"""Small fixed workloads for profiling one kernel (ncu -k ... -c 1).

    python -m paper_1110_6745_gb300.probe batch  [threads] [replicas]
        L = 2048 replicas (p = 0.95, q = 0.05: k = 32) through okz_batch_run:
        two runs of 8 sweeps each at the given CTA shape (default 512, 304).
    python -m paper_1110_6745_gb300.probe stream [L] [p] [q] [sweeps]
        one lattice through the parity stream kernel with the library's
        tiling (default L = 8192, p = 0.75, q = 0.25: k = 3, 24 sweeps).

Every launch of the chosen kernel does the same work, so a capture of one
launch past the first few describes them all.
"""
import sys

import paper_1110_6745_gb300 as okz


def batch(threads=512, replicas=304):
    L = [2048] * replicas
    with okz.Batch(L, [0.95] * replicas, [0.05] * replicas,
                   list(range(1, replicas + 1))) as b:
        b.set_tiling(threads, 32 * 1024)
        for _ in range(2):
            b.run([8] * replicas)
            b.sync()
    print("batch: %d x L = 2048, %d threads, 2 x 8 sweeps" % (replicas, threads))


def stream(L=8192, p=0.75, q=0.25, sweeps=24):
    with okz.Simulation(L, p, q, seed=31, kernel=okz.OKZ_KERNEL_PARITY_STREAM) as sim:
        sim.sweep(sweeps)
        sim.synchronize()
        print("stream: L = %d, p = %g, q = %g, %d sweeps, %d words per thread, %d sweeps per "
              "pass, band rows %d" % (L, p, q, sweeps, sim.wpt, sim.fuse, sim.band_rows))


def main(argv):
    okz.lib()
    if not argv or argv[0] not in ("batch", "stream"):
        print(__doc__)
        return 2
    if argv[0] == "batch":
        batch(*[int(a) for a in argv[1:3]])
    else:
        args = argv[1:5]
        conv = [int, float, float, int]
        stream(*[c(a) for c, a in zip(conv, args)])
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
