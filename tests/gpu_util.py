"""Shared helpers of the GPU parity tests (tolerances, comparisons, scene set-up)."""
import numpy as np

import oracle as O

# Tolerances, restating the targets the GPU path is held to:
#  - per pixel and channel |gpu - oracle| <= 1e-4 |oracle| + 1e-7 on >= 99.9 % of channels
#  - mean image error  mean|gpu - oracle| / mean|oracle| <= 1e-5
#  - interior gradient relative L2 <= 1e-3
PIX_REL, PIX_ABS, PIX_FRAC = 1e-4, 1e-7, 0.999
MEAN_REL = 1e-5
GRAD_REL = 1e-3


def image_report(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(gpu - ref)
    ok = err <= PIX_REL * np.abs(ref) + PIX_ABS
    mean_rel = err.mean() / max(np.abs(ref).mean(), 1e-30)
    return ok.mean(), mean_rel, err


def assert_image_parity(gpu, ref, frac=PIX_FRAC, mean_rel=MEAN_REL, what=""):
    f, m, err = image_report(gpu, ref)
    assert f >= frac and m <= mean_rel, "%s: %.5f of channels within tolerance, mean rel err %.2e, max err %.3e" % (
        what, f, m, err.max())


def rel_l2(got, exp):
    got = np.concatenate([np.asarray(g, np.float64).ravel() for g in got])
    exp = np.concatenate([np.asarray(e, np.float64).ravel() for e in exp])
    return np.linalg.norm(got - exp) / max(np.linalg.norm(exp), 1e-300)


def sample_pixels(sc, n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        vi = int(rng.integers(len(sc.views)))
        v = sc.views[vi]
        out.append((vi, int(rng.integers(v.width)), int(rng.integers(v.height))))
    return np.unique(np.array(out, np.int32), axis=0)


def oracle_pixels(sc, B, seed, pix, **kw):
    return O.render_pixels(O.OracleScene(sc), O.params(B, seed, **kw), pix)[0]
