"""One small filter call for kernel profiling (run under ncu).

  python -m paper_2005_09534_gb300.profile_step [F32|DF64|F64] [L] [n_b] [K]
  python -m paper_2005_09534_gb300.profile_step batched [F32|DF64] [n_inst] [K]

Filters a seeded block through P^K (sigma = 0) of the L-site XXZ chain with
W = 3 fields: K + 1 step-kernel launches per 128-byte column slice, so
`ncu -k regex:k_ham_step -s 3 -c 1` captures one full-size step launch.
The batched form filters n_inst L = 16 / 18 XXZ rings (n_b = 16) in one
cooperative launch of K steps (`ncu -k regex:k_filter_batched -c 1`).
"""
import sys

import torch

import polfed_inputs as I

from . import DF64, F32, F64, basis_build, cheb_filter, cheb_filter_batched, load


def batched(argv):
    kind = argv[2] if len(argv) > 2 else "DF64"
    n = int(argv[3]) if len(argv) > 3 else 16
    K = int(argv[4]) if len(argv) > 4 else 8
    dt = {"F32": (F32, torch.float32), "DF64": (DF64, torch.float64)}[kind]
    load()
    dev = torch.device("cuda:0")
    ms, Xs, Ys = [], [], []
    for r in range(n):
        L = 16 if r % 2 == 0 else 18
        m = I.xxz(L, 3.0, 3, r)
        dim = basis_build(L, L // 2)
        ms.append(m)
        Xs.append(torch.from_numpy(I.block(dim, 16, 100 + r)).to(dev, dt[1]))
        Ys.append(torch.empty_like(Xs[-1]))
    bound = [1.5 * (m.L * 0.75 + m.L * 1.5) for m in ms]  # > ||H||: bonds 3/4 each, fields |h_i|/2 <= 3/2
    cheb_filter_batched(ms, [-b for b in bound], bound, [0.0] * n, [K] * n, Xs, Ys, 16, dt[0])
    torch.cuda.synchronize()
    print("profile_step ok batched", kind, n, K)


def main(argv):
    if len(argv) > 1 and argv[1] == "batched":
        return batched(argv)
    kind = argv[1] if len(argv) > 1 else "F32"
    L = int(argv[2]) if len(argv) > 2 else 22
    nb = int(argv[3]) if len(argv) > 3 else 64
    K = int(argv[4]) if len(argv) > 4 else 6
    dt = {"F32": (F32, torch.float32), "DF64": (DF64, torch.float64), "F64": (F64, torch.float64)}[kind]
    load()
    dev = torch.device("cuda:0")
    m = I.xxz(L, 3.0, 4, 0)
    dim = basis_build(L, L // 2)
    st = torch.empty(dim, dtype=torch.int32, device=dev)
    basis_build(L, L // 2, st)
    X = torch.from_numpy(I.block(dim, nb, 7)).to(dev, dt[1])
    Y = torch.empty_like(X)
    bound = 1.5 * (L * 1.25 + L * 3.0 / 2)  # > ||H|| (each bond term <= 3/4, each field term <= 3/2)
    cheb_filter(m, st, dim, -bound, bound, 0.0, K, X, Y, nb, dt[0])
    torch.cuda.synchronize()
    print("profile_step ok", kind, L, dim, nb, K)


if __name__ == "__main__":
    main(sys.argv)
