"""The per-hop latency microbenchmark (vDebugHopLatency): a ring of CTAs on
chosen SMs, or one cluster, passes one FIFO line per protocol; it returns a
positive time per hop and the SM of each ring position, and refuses invalid
rings without launching."""
import pytest

from paper_2507_04786_b300 import VcommError
from paper_2507_04786_b300.binding import debug_hop_latency

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("proto", ["simple", "ll", "ll128"])
def test_ring_on_chosen_sms(proto):
    sms = [0, 1, 2, 3, 5]
    ns, got = debug_hop_latency(proto, sms, laps=200)
    assert got == sms
    assert 0 < ns < 1e6


@pytest.mark.parametrize("proto", ["ll", "ll128"])
def test_ring_as_one_cluster(proto):
    ns, got = debug_hop_latency(proto, None, n=8, laps=200)
    assert 0 < ns < 1e6
    assert len(set(got)) == 8 and min(got) >= 0


@pytest.mark.parametrize("sms,n", [([0], 0), ([0, 0], 0), ([0, 5000], 0), (None, 17), (None, 1)])
def test_invalid_rings_are_refused(sms, n):
    with pytest.raises(VcommError) as e:
        debug_hop_latency("ll", sms, n=n, laps=10)
    assert e.value.name == "vInvalidArgument"
