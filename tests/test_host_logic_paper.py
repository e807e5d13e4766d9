"""Host logic without a GPU: the adaptive-rank controller's decisions (against a
stand-in batch with prescribed spectra) and the paper workload's flop count."""
import numpy as np

import paper_2508_18114_gb300.adaptive as adaptive


class FakeBatch:
    """Stands in for LowRankBatch: records the calls; the spectrum of trajectory
    tj at record r is p_1 = 1, p_M = script[r][tj // 2]."""
    log = []

    def __init__(self, models, ranks, script, **kw):
        self.ranks = list(ranks)
        self.script = script
        self.step = 0
        self.n = len(models)

    def set_pulse(self, pulses, tau):
        FakeBatch.log.append(("pulse", tau))

    def set_initial(self, seed, eps):
        FakeBatch.log.append(("initial", seed, eps))

    def integrate(self, dt, k):
        self.step += k
        FakeBatch.log.append(("integrate", self.step))

    def diagnostics(self):
        nrec = len(self.script) + 1
        M = max(self.ranks)
        eig = np.zeros((2 * self.n, nrec, M))
        for r, row in enumerate(self.script, start=1):
            for tj in range(2 * self.n):
                c = tj // 2
                eig[tj, r, 0] = 1.0
                eig[tj, r, self.ranks[c] - 1] = row[c]
        return None, eig

    def grown(self, ranks, seed, eps):
        FakeBatch.log.append(("grow", list(ranks), seed, eps))
        b = FakeBatch([None] * self.n, ranks, self.script)
        b.step = self.step
        return b


def test_controller_grows_above_tol_up_to_max(monkeypatch):
    script = [[0.5, 1e-6], [1e-6, 2e-3], [5e-3, 5e-3], [1.0, 1.0]]
    FakeBatch.log = []
    monkeypatch.setattr(adaptive, "LowRankBatch",
                        lambda models, ranks, **kw: FakeBatch(models, ranks, script, **kw))
    b, hist = adaptive.adaptive_run([0, 0], [None, None], 1.0, 1e-3, 400, rank0=2, max_rank=5, d_rank=2,
                                    tol=1e-3, segment=100, seed=3, eps=1e-5, grow_seed=10)
    assert [h["ranks"] for h in hist] == [[4, 2], [4, 4], [5, 5], [5, 5]]
    grows = [x for x in FakeBatch.log if x[0] == "grow"]
    assert grows == [("grow", [4, 2], 10, 1e-5), ("grow", [4, 4], 11, 1e-5), ("grow", [5, 5], 12, 1e-5)]
    assert [h["step"] for h in hist] == [100, 200, 300, 400]
    assert b.ranks == [5, 5]


def test_controller_stops_deciding_after_a_partial_segment(monkeypatch):
    script = [[0.5], [0.5]]
    FakeBatch.log = []
    monkeypatch.setattr(adaptive, "LowRankBatch",
                        lambda models, ranks, **kw: FakeBatch(models, ranks, script, **kw))
    _, hist = adaptive.adaptive_run([0], [None], 1.0, 1e-3, 150, rank0=2, max_rank=8, d_rank=2, tol=1e-3,
                                    segment=100)
    assert [h["step"] for h in hist] == [100]
    assert [x for x in FakeBatch.log if x[0] == "integrate"][-1] == ("integrate", 150)


def test_paper_flop_count_matches_a_hand_count():
    import bench
    N, M, K = 10, 3, 2
    rowptr = np.array([0, 2, 4, 6, 8, 10, 12, 14, 16, 18, 20] +       # A: 2 per row
                      [20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30] +   # L_1: 1 per row
                      [30] * 11 +                                      # L_2: empty
                      [30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40])    # r (not counted)
    model = {"N": N, "n_jumps": K, "rowptr": rowptr}
    entries = 30
    want = 8 * entries * M + 8 * N * (M * (M + 1) // 2 + K * M * M) + 8 * K * N * M * M + 12 * N * M
    assert bench.paper_flops_per_stage(model, M) == want
