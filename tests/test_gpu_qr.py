"""The final QR step of Algorithm 1 (Section 3.4) on the GPU against the oracle's: the same
orthonormal factors, transformed core and coupled factors (FP64 arithmetic on both sides,
FP32 storage on the GPU: 1e-5 relative to each block's largest entry), unchanged
predictions, and the rank-deficiency error."""
import numpy as np
import pytest

from paper_1708_08640_gb300 import synth
from tests.gpu_common import make_pair

pytestmark = pytest.mark.gpu


def as_np(t):
    return t.detach().cpu().double().numpy()


def close(got, ref, tol, what):
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    err = np.max(np.abs(got - ref))
    scale = np.max(np.abs(ref))
    assert err <= tol * scale, f"{what}: max error {err:.3e} vs largest entry {scale:.3e}"


@pytest.mark.parametrize("name", ["cfg0", "cfg1_tiny", "cfg3_tiny"])
def test_finalize_qr_matches_oracle(cuda_lib, name):
    p = synth.make_problem(name)
    gpu, orc, q, order = make_pair(p)        # the seeded initial parameters
    G, U, V = gpu.get_params()
    orc.set_params(as_np(G), [as_np(u) for u in U], [as_np(v) for v in V])
    test_idx = np.ascontiguousarray(q.test_idx, dtype=np.int32)
    before = as_np(gpu.predict(test_idx))
    cpl_before = [orc.predict_coupled(m, c.rows, c.cols) for m, c in enumerate(q.coupled)]
    gpu.finalize_qr()
    orc.finalize_qr()
    G1, U1, V1 = gpu.get_params()
    close(as_np(G1), orc.G, 1e-5, "G")
    for n, u in enumerate(U1):
        close(as_np(u), orc.U[n], 1e-5, f"U{n}")
        uu = as_np(u)
        close(uu.T @ uu, np.eye(uu.shape[1]), 1e-5, f"U{n}^T U{n}")
    for m, v in enumerate(V1):
        close(as_np(v), orc.V[m], 1e-5, f"V{m}")
    close(as_np(gpu.predict(test_idx)), before, 1e-5, "tensor predictions")
    orc.set_params(as_np(G1), [as_np(u) for u in U1], [as_np(v) for v in V1])
    for m, c in enumerate(q.coupled):
        close(orc.predict_coupled(m, c.rows, c.cols), cpl_before[m], 1e-5, f"coupled {m}")
    gpu.close()


def test_finalize_qr_rejects_rank_deficient_factor(cuda_lib):
    from paper_1708_08640_gb300._lib import S3Error
    p = synth.make_problem("cfg0")
    gpu, orc, q, order = make_pair(p)
    G, U, V = gpu.get_params()
    U = [as_np(u) for u in U]
    U[1][:, 3] = U[1][:, 1]                    # dependent columns
    gpu.set_params(as_np(G), U, [as_np(v) for v in V])
    with pytest.raises(S3Error):
        gpu.finalize_qr()
    G2, U2, _ = gpu.get_params()               # nothing changed
    np.testing.assert_array_equal(as_np(U2[1]), U[1].astype(np.float32).astype(np.float64))
    np.testing.assert_array_equal(as_np(G2), as_np(G))
    gpu.close()
