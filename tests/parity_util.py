"""The parity rule lives beside the oracle (oracle/parity.py) so that the
smoke check and the benchmark's parity report apply the same rule."""
from oracle.parity import *  # noqa: F401,F403
from oracle.parity import _per_record  # noqa: F401
