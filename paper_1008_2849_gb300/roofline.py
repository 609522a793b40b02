"""Algorithmic byte model of the sort (what a pass must move, at minimum).

Every counting-sort pass reads each item once and writes it once (Sec. 3);
an item is a 4-byte key, plus a 4-byte value for key-value sorts (Sec. 1).
Sec. 5 counts the writes of a 64 Mi-pair sort as 64 Mi x 8 B x 4 passes.
The one up-front histogram read adds 4 bytes per key.  Look-back status
words and other bookkeeping are overhead, not algorithmic bytes.
"""

KEY_BYTES = 4
VALUE_BYTES = 4
PASSES = 4


def item_bytes(with_values: bool) -> int:
    return KEY_BYTES + (VALUE_BYTES if with_values else 0)


def scatter_bytes_per_item(with_values: bool) -> int:
    """Bytes one scatter pass moves per item: one read plus one write."""
    return 2 * item_bytes(with_values)


def histogram_bytes_per_item() -> int:
    """Bytes the up-front histogram moves per item: one key read."""
    return KEY_BYTES


def sort_bytes_per_item(with_values: bool, passes: int = PASSES) -> int:
    """Histogram read plus ``passes`` scatter passes."""
    return histogram_bytes_per_item() + passes * scatter_bytes_per_item(with_values)
