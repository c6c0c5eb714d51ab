"""The issue-rate probe behind the evaluation ceiling of the roofline: every
kind returns a rate inside what an SM can issue (4 schedulers x 32 lanes of
instructions per clock), and packed or three-input forms count two element
operations per instruction."""
import pytest

from paper_2511_15629_b300 import esdp as E

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", range(len(E.ALU_PROBE_KINDS)))
def test_alu_probe_rates_are_physical(kind):
    ins, elem = E.alu_probe(kind, 512)
    assert 8.0 <= ins <= 128.0 * 1.02
    assert elem == pytest.approx(ins * (2.0 if kind in (1, 3) else 1.0))


def test_alu_probe_rejects_bad_kind():
    with pytest.raises(E.EsdpError):
        E.alu_probe(7, 16)
