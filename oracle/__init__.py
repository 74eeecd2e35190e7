"""CPU FP64 oracle of the confined TTSH solver: test infrastructure, never on the product path."""
