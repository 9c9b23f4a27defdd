"""Argument checks of the Python binding that run before any library call:
buffers whose size differs from what the C entry point will read or write
are refused on the host (a wrong size would otherwise reach the device as an
out-of-bounds access)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2407_10797_gb300 import fstat  # noqa: E402


def fake_mlp(groups, P=10):
    """An MLP object without a device network: only the host checks run."""
    m = fstat.MLP.__new__(fstat.MLP)
    m.groups, m.P, m.width, m._L, m._h, m.stream = groups, P, 8, None, None, None
    return m


@pytest.mark.parametrize("groups", [1, 3])
def test_parameter_vector_length(groups):
    m = fake_mlp(groups)
    with pytest.raises(ValueError):
        m.set_params(torch.zeros(groups * m.P - 1))
    with pytest.raises(ValueError):
        m.set_params(torch.zeros(groups * m.P + 1))


def test_single_network_shapes():
    m = fake_mlp(1)
    with pytest.raises(ValueError):
        m.forward(torch.zeros(4, 6))                       # rows of 6
    with pytest.raises(ValueError):
        m.forward(torch.zeros(4, 5), y=torch.zeros(3))     # output too short
    with pytest.raises(ValueError):
        m.loss_grad(torch.zeros(4, 5), torch.zeros(5))     # one target too many
    with pytest.raises(ValueError):
        m.train(torch.zeros(4, 5), torch.zeros(3), 1)


def test_network_batch_shapes():
    m = fake_mlp(2)
    with pytest.raises(ValueError):
        m.forward(torch.zeros(4, 5))                       # not [G][N][5]
    with pytest.raises(ValueError):
        m.forward(torch.zeros(3, 4, 5))                    # 3 blocks for 2 networks
    with pytest.raises(ValueError):
        m.forward(torch.zeros(2, 4, 5), y=torch.zeros(7))
    with pytest.raises(ValueError):
        m.train(torch.zeros(2, 4, 5), torch.zeros(2, 5), 1)


def test_noalloc_wrapper_checks_sizes_against_the_grid():
    from paper_2407_10797_gb300 import synth as S
    g = S.tiny_grid(n=100, f_min=0.02, stride=8)
    d = torch.zeros(g.n, dtype=torch.complex128)
    psd = torch.ones(g.n, dtype=torch.float64)
    P = torch.zeros(4, 6, dtype=torch.float64)
    with pytest.raises(ValueError):
        fstat.fstat_batch_noalloc(g, d[:-1], psd, P, 2)                 # one bin short
    with pytest.raises(ValueError):
        fstat.fstat_batch_noalloc(g, d, psd[:-1], P, 2)
    with pytest.raises(ValueError):
        fstat.fstat_batch_noalloc(g, d, psd, P[:, :5], 2)               # params [B, 5]
    with pytest.raises(ValueError):
        fstat.fstat_batch_noalloc(g, d, psd, P, 2, F=torch.zeros(3, dtype=torch.float64))
    with pytest.raises(ValueError):
        fstat.fstat_batch_noalloc(g, d, psd, P, 2, F=torch.zeros(4, dtype=torch.float64),
                                  F_part=torch.zeros(4, 3, dtype=torch.float64))


def test_missing_library_is_an_error_not_a_fallback():
    """Without the CUDA library the binding raises: there is no CPU path to
    fall back to (run in a child process so the loaded library of this
    session is not disturbed)."""
    import os
    import subprocess
    import sys
    code = ("import paper_2407_10797_gb300.build as b\n"
            "b.LIB = '/nonexistent/libfs_gb300.so'\n"
            "b.up_to_date = lambda: True\n"
            "from paper_2407_10797_gb300 import fstat\n"
            "for call in (lambda: fstat.load(build_if_missing=False),\n"
            "             lambda: fstat.Plan(100, 0.01, 1e-6, 1e7)):\n"
            "    try:\n"
            "        call()\n"
            "        print('loaded')\n"
            "    except ImportError as e:\n"
            "        print('refused', 'missing' in str(e))\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.split() == ["refused", "True", "refused", "True"], r.stdout
