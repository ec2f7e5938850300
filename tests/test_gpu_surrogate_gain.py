"""What the trained surrogate gains over the plain method, judged by the plain method.

A surrogate trained on residual spectra of the batched method answers part of the held-out
queries; for those its RV must agree with the plain method's within 10 cm/s (up to the 1%
calibration miss rate plus sampling slack), and answering them must be cheaper per query than
the plain method.  The measured gain and acceptance are printed."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_04259_gb300 import soap
    return soap


def test_surrogate_gain_over_the_plain_method(S):
    from paper_2301_04259_gb300 import synth
    from paper_2301_04259_gb300 import surrogate_pipeline as SP
    case = synth.batch_spectra(0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    with S.Disk(case.star, t(case.quiet), {k: t(v) for k, v in case.active.items()}) as d:
        model = SP.train(d.ctx, case, n_train=300_000, epochs=100, n_judge=98_304, judge_epochs=60, seed=3)
        try:
            xe = synth.surrogate_params(1234, 8192)
            err = SP.judge_errors(d.ctx, case, model, xe)
            acc = torch.empty(len(xe), dtype=torch.uint8, device=DEV)
            S.soap_surrogate_predict(model.handle, t(xe), model.accept_thr_cms, accepted=acc)
            a = acc.cpu().numpy().astype(bool)
            assert a.mean() >= 0.05, a.mean()
            assert (err[a] > SP.RV_ERR_MAX_CMS).mean() <= 0.03
            # per-query cost of what the surrogate answers vs the plain method on the same queries
            n_px = case.star.n_px
            xa = xe[a]
            out = torch.empty((len(xa), n_px), dtype=torch.float32, device=DEV)
            coef = torch.empty((len(xa), 128), dtype=torch.float32, device=DEV)
            xad = t(xa)

            def surrogate():
                S.soap_surrogate_predict(model.handle, xad, model.accept_thr_cms, coef=coef)
                S.soap_surrogate_reconstruct(model.handle, coef, out)

            def plain():
                SP.plain_residuals(d.ctx, xa, out)

            times = {}
            for name, fn in (("surrogate", surrogate), ("plain", plain)):
                fn()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(3):
                    fn()
                torch.cuda.synchronize()
                times[name] = (time.perf_counter() - t0) / 3
            gain = times["plain"] / times["surrogate"]
            print(f"accepted {a.mean():.3f}, accepted RV err p99 {np.percentile(err[a], 99):.2f} cm/s, "
                  f"per-query gain on accepted queries {gain:.2f}x, hybrid gain "
                  f"{1.0 / (1.0 - a.mean() + a.mean() / gain):.3f}x")
            assert gain > 1.5
        finally:
            model.free()
