"""The named synthetic workloads (sizes and seeds fixed here).

Each stands in for one class of the paper's social and information networks
(Table 1), which are not available: heavy-tailed degree distributions, a dense
core and one large clique planted at uniformly random vertices.
"""
from __future__ import annotations

from . import Batch, Graph, chung_lu, er_batch, rmat

CHUNG_LU_20K = "chung-lu n=20000 gamma=2.5 mean=8 cap=1000 planted=15 seed=1"
RMAT_S22 = "rmat scale=22 ef=16 abc=(0.57,0.19,0.19) planted=40 seed=2"
ER_BATCH_4096 = "er-batch count=4096 n~U[64,4096] d~U[8,64] planted~U[8,24] seed=3"
RMAT_S24 = "rmat scale=24 ef=16 abc=(0.57,0.19,0.19) planted=60 seed=4"
CHUNG_LU_100M = "chung-lu n=100000000 gamma=2.1 mean=36 cap=10000 planted=80 seed=5"


def chung_lu_20k() -> Graph:
    return chung_lu(20000, 2.5, 8.0, 1000.0, planted=15, seed=1)


def rmat_s22() -> Graph:
    return rmat(22, 16, 0.57, 0.19, 0.19, planted=40, seed=2)


def er_batch_4096(count: int = 4096) -> Batch:
    return er_batch(count, seed=3)


def rmat_s24() -> Graph:
    return rmat(24, 16, 0.57, 0.19, 0.19, planted=60, seed=4)


def chung_lu_100m() -> Graph:
    return chung_lu(100_000_000, 2.1, 36.0, 10000.0, planted=80, seed=5)


BY_NAME = {
    CHUNG_LU_20K: chung_lu_20k,
    RMAT_S22: rmat_s22,
    ER_BATCH_4096: er_batch_4096,
    RMAT_S24: rmat_s24,
    CHUNG_LU_100M: chung_lu_100m,
}
