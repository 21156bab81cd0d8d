"""x-slab decomposition on the GPU (Sec. 4.3 ghost-layer exchange): two
processes share cuda:0, each stepping one slab with halo columns that the
library's pack / unpack kernels exchange after every step (carried through
gloo on the host); the gathered slabs equal the whole-lattice run to
rounding, within 1e-12 of each field's magnitude (FP64; walls with a moving
top wall and a contact angle, periodic RK4 with its 5-column halo, and a wide
lattice on the tiled kernel).  The kernels never wait on one another: every
exchange is host-synchronised."""
import os
import socket
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("name", ["d3q7_walls_moving", "rk4_periodic", "d3q19_wide_tiled"])
def test_x_slabs_equal_whole_lattice(name, tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_03041_gb300 import build
    build.build()
    port = _free_port()
    out = str(tmp_path / "result.txt")
    procs = [subprocess.Popen([sys.executable, os.path.join(HERE, "slab_worker.py"), str(r), "2", str(port),
                               name, "12", out], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
             for r in range(2)]
    logs = []
    for p in procs:
        o, _ = p.communicate(timeout=600)
        logs.append(o)
        assert p.returncode == 0, "\n".join(logs)
    assert open(out).read().strip() == "ok", open(out).read()
