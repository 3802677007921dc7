"""The profiling sweep (one call of every entry point) runs on small meshes
and leaves the device status clean."""
import pytest

from paper_2602_12365_b300 import sweep

pytestmark = pytest.mark.gpu


def test_sweep_small_meshes():
    sweep.tet_sweep(4)
    sweep.hex_sweep(3)
